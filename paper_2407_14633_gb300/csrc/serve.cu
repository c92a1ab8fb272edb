// Serving: continuous batching of self-consistent solves (filled in below).
#include "ctx.h"

namespace negf {
struct Serve {};
void serve_free(Ctx* c) {
  delete c->serve;
  c->serve = nullptr;
}
}  // namespace negf
