// Declarations of the sweep of 1 x 1 chains split along the channel (sweep_seg.cu) and of its
// plan structures (built in compute.cu).
#pragma once
#include "common.cuh"

namespace negf {

// Sweep of a 1 x 1 chain split along the channel (sweep_seg.cu): segments of SEG_LEN layers, one
// warp per (item, segment).  Used for FP64 items of devices with at least SEG_MIN_L layers and
// at most SEG_MAX_ITEMS such items of their own.
constexpr int SEG_LEN = 512;
constexpr int SEG_MIN_L = 16384;
constexpr int SEG_MAX_ITEMS = 128;
constexpr int SEG_FIELDS = 21;     // doubles per lane of a segment record
struct SegItem {
  int item;        // index into the plan's WorkItem array
  int n_seg;       // ceil(L / SEG_LEN)
  long long rec0;  // first record of the item (within its wave)
  long long stage; // byte offset of its staging (within its wave)
};
struct SegArgs {
  const DeviceView* devs;
  const WorkItem* items;
  const SegItem* segs;     // the wave's items
  const int* rec_item;     // per record of the wave: index into segs
  long long n_rec;
  int n_segitems;
  double* rec;             // SEG_FIELDS x 32 doubles per record
  unsigned char* stage;    // per item: L x (3 real axis | 2 contour) x 32 doubles
  double* partial;
  double* Tpart;
  double* ring_cap;
  int cap_ring;
};
size_t seg_stage_bytes(int L, int kind);
// the five launches of one wave
int launch_seg(const SegArgs& a, cudaStream_t s);

}  // namespace negf
