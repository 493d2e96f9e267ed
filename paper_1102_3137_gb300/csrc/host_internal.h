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

// A plan's device buffers, for host code that composes solves (the recursive
// decomposition): the staged inputs a solve reads (omega [K], V [N], sigma
// complex[K][N], q1 [N]) and the results of the last solve in the
// subdomain-first layout (acc = diag(Q T Q^T) and diagB = diag(B^-1), both
// complex[K][Ndd]; dd2nat maps a slot to its natural site, -1 on padding;
// status [K] the DYSON_ST_* flags).
struct PlanDev {
  double* omega;
  double* V;
  double* sigma;
  double* q1;
  const double* acc;
  const double* diagB;
  const int* dd2nat;
  const int* status;
  int Ndd;
  int N;
};
int dyson_internal_plan_dev(dyson_plan_s* p, PlanDev* out);
// the whole solve on inputs already in the plan's buffers (no copies in or out)
int dyson_internal_solve_resident(dyson_plan_s* p, int K, void* stream);
// the subdomain factorization alone on staged inputs (diagB; exact when p = 1)
int dyson_internal_factor_resident(dyson_plan_s* p, int K, void* stream);
