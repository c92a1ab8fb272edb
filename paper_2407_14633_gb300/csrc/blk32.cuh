// Host entry points of the register-tiled complex64 sweep of wide ring blocks
// (sweep_block32.cu).
#pragma once
#include "common.cuh"

namespace negf {

// Tile class (CTA width in warps: 1, 2 or 4) that runs blocks of width b with leads of m
// sites at a requested width: the smallest class holding b x b that is at least that wide;
// 0 when no class holds b (b > 36) or m > b.
int blk32_class(int b, int m, int warps);
size_t blk32_smem_bytes(int nw);
// staging bytes per layer of one lane (gL_l and R_l tiles)
long long blk32_stage_layer_bytes(int nw);
// whether a lane of blocks b x b with leads of m sites can be re-swept in FP64 inside a CTA of
// class nw (the FP64 compact layout at that width fits the class's shared memory)
bool blk32_can_fuse(int b, int m, int nw);
// resident CTAs per SM and launch, without (fuse = 0) or with the in-CTA FP64 re-sweep of
// flagged lanes (a.fuse = 1; dynamic shared memory as the class's)
int blk32_occupancy(int nw, int fuse);
int launch_blk32(const SweepArgs& a, int grid, int nw, cudaStream_t s);

}  // namespace negf
