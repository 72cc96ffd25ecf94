// finalize.cuh -- end-of-step work shared by the standalone finalisation
// kernel and the particle kernel (which runs it after its last sub-step):
// the step's sums go into the compensated time sums and the protocol
// advances to the next step.
#pragma once

#include "susp_dev.cuh"

namespace susp_dev {

// Compensated time sums per box: 47 entries (and their compensations).
constexpr int NSUMS = 47;

__device__ __forceinline__ void proto_derive(Proto& s, int nx) {
  const double dm = s.delta - nx * floor(s.delta / nx);
  s.di = (int)floor(dm);
  s.w = dm - s.di;
  s.near_lo = (s.w < 0.5) ? 0 : 1;
  s.near_hi = ((1.0 - s.w) < 0.5) ? 0 : 1;
  s.wf_lo = (float)s.w;
  s.wf_hi = (float)(1.0 - s.w);
  s.delta_f = (float)s.delta;
  s.ule_f = (float)s.ule;
}

__device__ __forceinline__ void kahan_le(double& delta, double& comp, double inc, int nx) {
  const double y = inc - comp;
  const double t = delta + y;
  comp = (t - delta) - y;
  delta = t;
  if (delta >= nx) delta -= nx;
  if (delta < 0.0) delta += nx;
}

// End of step t, one block per box: the step's sums (accumulated by the
// collide-stream, boundary-link and particle kernels) go into the compensated
// time sums and are cleared; then the protocol advances to t+1.
// Call with every thread of a block of at least 64 threads (it has block
// barriers); the protocol is advanced by thread 0.
static __device__ __noinline__ void finalize_box(const View& v) {
  __shared__ double tot[40];
  // The kernel is a short chain of dependent memory round trips; every
  // address and every operand that does not depend on the replica sums is
  // loaded before the barrier so those trips overlap.
  const int k = threadIdx.x;
  double* const a = v.step_acc + k;
  double* const S = v.sums;
  Proto* const pp = v.proto;
  const bool move = v.move != 0;
  unsigned long long* const counters = v.counters;
  const int nx = v.nx;
  double s_k = 0.0, c_k = 0.0;
  if (k < NSUMS) { s_k = S[k]; c_k = S[NSUMS + k]; }
  Proto s;
  double ule_nn = 0.0;   // shear increment of step t+2 -> t+3 (needs only the protocol constants)
  if (k == 0) { s = *pp; ule_nn = proto_increment(s, s.t + 2); }
  // phase of this step for Eq. 17, 18: the step t -> t+1 shears by
  // gamma(t+1) - gamma(t), so its stress belongs to omega (t + 1/2) + Theta
  // (read before thread 0 advances the protocol below)
  double cs = 0.0;
  if (k == 45 || k == 46) {
    const int kind = pp->kind;
    const double om = kind == 1 ? pp->omega : 0.0, th0 = kind == 1 ? pp->theta : 0.0;
    const double phase = om * ((double)pp->t + 0.5) + th0;
    cs = k == 45 ? cos(phase) : sin(phase);
  }
  // 0-5 viscous, 6-14 stresslet, 15-23 contact virial, 24 contact count,
  // 25-33 repulsive virial, 34-39 lubrication stresslets (xx yy zz xy xz yz);
  // the replicas added in a fixed order, then cleared
  if (k < 40) {
    double part[ACC_REP];
#pragma unroll
    for (int r = 0; r < ACC_REP; ++r) part[r] = a[r * ACC_STRIDE];   // loads issued together
    double x = 0.0;
#pragma unroll
    for (int r = 0; r < ACC_REP; ++r) {
      x += part[r];
      a[r * ACC_STRIDE] = 0.0;
    }
    tot[k] = x;
  }
  __syncthreads();
  if (k < NSUMS) {
    // compensated time sums, one entry per thread; the viscous and
    // lubrication partials are xx yy zz xy xz yz, expanded to the full
    // 3 x 3; entries 45 and 46: the step's total shear stress sigma_xy
    // (times V; stresslet symmetrised, virials with a minus) weighted by cos
    // and sin of the phase
    const int vmap[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
    double x;
    if (k < 9) x = tot[vmap[k]];
    else if (k < 18) x = tot[6 + (k - 9)];
    else if (k < 27) x = move ? tot[15 + (k - 18)] : 0.0;
    else if (k < 36) x = move ? tot[25 + (k - 27)] : 0.0;
    else if (k < 45) x = move ? tot[34 + vmap[k - 36]] : 0.0;
    else {
      const double sxy = tot[3] + 0.5 * (tot[7] + tot[9]) - (move ? tot[16] + tot[26] - tot[37] : 0.0);
      x = sxy * cs;
    }
    const double y = x - c_k;
    const double t = s_k + y;
    S[NSUMS + k] = (t - s_k) - y;
    S[k] = t;
  }
  if (k != 0) return;
  counters[0] += 1ULL;
  if (move) counters[1] += (unsigned long long)(tot[24] + 0.5);
  // protocol: t -> t+1
  s.t += 1;
  s.delta = s.delta_n; s.delta_c = s.delta_nc; s.ule = s.ule_n;
  s.delta_n = s.delta; s.delta_nc = s.delta_c;
  kahan_le(s.delta_n, s.delta_nc, s.ule, nx);
  s.ule_n = ule_nn;
  proto_derive(s, nx);
  *pp = s;
}


}  // namespace susp_dev
