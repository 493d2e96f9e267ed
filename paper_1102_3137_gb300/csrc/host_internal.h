// Host-side entry points shared by the C ABI (api.cu) and the serving loop
// (server.cu) that device code never sees.
#pragma once

struct dyson_plan_s;

// One request's share of a fused solve: K frequencies with their own omega,
// sigma and outputs; V and q1 are shared by every segment.
struct SolveSeg {
  int K;
  const double* omega;
  const double* sigma;
  double* diagG;
  int* status;
};
// dyson_internal_solve_enqueue over several segments solved as one batch of
// sum(K) frequencies (their omega and sigma staged side by side, each
// segment's outputs copied back to its own buffers)
int dyson_internal_solve_enqueue_segs(dyson_plan_s* p, int nseg, const SolveSeg* segs, const double* V,
                                      const double* q1, int mem_kind, void* stream);
