// dem.cu — particle sub-steps: cell list, pair interactions, integration.
//
// Pair interactions (one warp per particle over its candidate partners,
// collected once per lattice step from the 27 cells around it; every pair is
// evaluated by both partners in the canonical orientation a = min(i, j),
// b = max(i, j) so the two results are bitwise equal and opposite, with no
// atomics):
//   contact (Sec. 2, Eq. 11, 11t): F_n = kn delta_n + eta_n v_n along -n,
//     tangential spring delta_t (kept per pair in a table owned by a),
//     projected onto the tangent plane and advanced by v_t dt, F_t = -kt delta_t
//     capped at mu |F_n| (Coulomb slip, spring reset to the slip length),
//     torques a_a n x F_t and a_b n x F_t;
//   double-layer repulsion F0 exp(-h / debye) (Eq. 13);
//   lubrication correction (Appendix A) with the leading-order X^A, Y^A,
//     Y^B, Y^C functions, beta = a_b / a_a, roughness delta, minus the value
//     at the cutoff gap.
// Lees-Edwards minimum image: d = R_b - R_a, k = round(d_y / L_y),
// d -= k (Delta, L_y, 0), and b's image moves with U_b + k U_LE e_x.
// Integration (Eq. 1): semi-implicit Euler with the hydrodynamic link force
// held over the sub-steps; Lees-Edwards wrap of the centres at the end.
// Driven spheres (the bumpy walls of Sec. 3) keep their velocity and spin:
// only their centres advance, and a Lees-Edwards crossing leaves their
// velocity as it is.
#include <cooperative_groups.h>

#include "susp_dev.cuh"
#include "finalize.cuh"

namespace susp_dev {

__global__ void k_cell_count(Batch B) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B.part_off[B.nbox]) return;
  const int bx = box_of(B.part_off, B.nbox, g);
  const View& v = B.views[bx];
  if (v.brute || !v.move) return;
  const int i = g - B.part_off[bx];
  double x = v.R[3 * i], y = v.R[3 * i + 1], z = v.R[3 * i + 2];
  x -= v.nx * floor(x * v.inv_nx_d);
  z -= v.nz * floor(z * v.inv_nz_d);
  int cx = (int)floor(x * v.inv_csx), cy = (int)floor(y * v.inv_csy), cz = (int)floor(z * v.inv_csz);
  cx = min(max(cx, 0), v.ncx - 1);
  cy = min(max(cy, 0), v.ncy - 1);
  cz = min(max(cz, 0), v.ncz - 1);
  const int c = cx + v.ncx * (cy + v.ncy * cz);
  v.pcell[i] = c;
  atomicAdd(v.cell_cnt + c, 1);
  // cells searched around i during this step's sub-steps; the rows beyond the
  // Lees-Edwards planes are shifted by -/+ Delta
  const double delta = v.proto->delta;
  double xb = x + delta, xa = x - delta;
  xb -= v.nx * floor(xb * v.inv_nx_d);
  xa -= v.nx * floor(xa * v.inv_nx_d);
  int* pc = v.pcx + 8 * i;
  pc[0] = cx; pc[1] = cy; pc[2] = cz;
  pc[3] = min(max((int)floor(xb * v.inv_csx), 0), v.ncx - 1);
  pc[4] = min(max((int)floor(xa * v.inv_csx), 0), v.ncx - 1);
}

// Exclusive scan of one box's cell counts per block (1024 threads).
__global__ void k_cell_scan(Batch B) {
  __shared__ int part[1024];
  const View& v = B.views[blockIdx.x];
  if (v.brute || !v.move || v.n == 0) return;
  const int nc = v.ncells, T = blockDim.x, t = threadIdx.x;
  const int chunk = (nc + T - 1) / T;
  const int b0 = t * chunk, b1 = min(nc, b0 + chunk);
  int s = 0;
  for (int c = b0; c < b1; ++c) s += v.cell_cnt[c];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const int add = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  int run = t ? part[t - 1] : 0;
  for (int c = b0; c < b1; ++c) {
    const int cnt = v.cell_cnt[c];
    v.cell_start[c] = run;
    run += cnt;
    v.cell_cnt[c] = 0;
  }
  if (t == T - 1) v.cell_start[nc] = part[T - 1];
}

__global__ void k_cell_fill(Batch B) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B.part_off[B.nbox]) return;
  const int bx = box_of(B.part_off, B.nbox, g);
  const View& v = B.views[bx];
  if (v.brute || !v.move) return;
  const int i = g - B.part_off[bx];
  const int c = v.pcell[i];
  const int slot = atomicAdd(v.cell_cnt + c, 1);
  v.cell_ids[v.cell_start[c] + slot] = i;
}

// Sort each cell's ids ascending so the gather order is deterministic; the
// counts are cleared for the next step's count.
__global__ void k_cell_sort(Batch B) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B.cell_off[B.nbox]) return;
  const int bx = box_of(B.cell_off, B.nbox, g);
  const View& v = B.views[bx];
  if (v.brute || !v.move) return;
  const int c = g - B.cell_off[bx];
  const int s = v.cell_start[c], e = v.cell_start[c + 1];
  for (int a = s + 1; a < e; ++a) {
    const int key = v.cell_ids[a];
    int b = a - 1;
    while (b >= s && v.cell_ids[b] > key) { v.cell_ids[b + 1] = v.cell_ids[b]; --b; }
    v.cell_ids[b + 1] = key;
  }
  v.cell_cnt[c] = 0;
}

template <typename T>
__device__ inline void cross3(const T a[3], const T b[3], T o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
__device__ inline T dot3(const T a[3], const T b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <typename T>
struct PairOut {
  T Fa[3], Ta[3], Tb[3];   // total pair force on a (b gets -Fa), torques on a and b
  T Fc[3];                 // contact part of Fa (for the virial)
  T Fr[3];                 // double-layer part of Fa
  T ht[3];                 // updated tangential spring
  T fn;                    // normal-force magnitude (repulsive positive)
  T S[6];                  // lubrication stresslet S_a + S_b (xx yy zz xy xz yz), when asked for
  T d[3];                  // R_b - R_a (minimum image)
  int touching;
};

template <typename T>
__device__ __forceinline__ void load_pair_const(const View& v, PairConst<T>& c) {
  if constexpr (sizeof(T) == 8) c = v.pc_d;
  else c = v.pc_f;
}

// Minimum-image displacement R_b - R_a and gap h = |d| - (a_a + a_b) of the
// pair (a, b) in FP64 (the FP32 compute path takes them from the step
// constants instead, see pairs_of); false when the pair is out of range.
template <typename T>
__device__ inline bool pair_geometry(const View& v, const double* Rs, int a, int b, T delta,
                                     const PairConst<T>& pc, T d[3], int& k, T& h) {
  static_assert(sizeof(T) == 8, "FP64 path");
  const T* pl = reinterpret_cast<const T*>(v.plb);
  const T rsum = pl[12 * a + 9] + pl[12 * b + 9];
  const T lim = rsum + pc.hrange + (T)1e-6;
  d[0] = Rs[3 * b] - Rs[3 * a];
  d[1] = Rs[3 * b + 1] - Rs[3 * a + 1];
  d[2] = Rs[3 * b + 2] - Rs[3 * a + 2];
  k = le_image<T>(d[0], d[1], d[2], delta, v.nx, v.ny, v.nz, v.inv_nx_d, v.inv_ny_d, v.inv_nz_d);
  const T d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (!(d2 < lim * lim)) return false;   // cheap rejection before the square root
  h = sqrt(d2) - rsum;
  return (h < pc.hrange) || (h < (T)0);
}

// uab = U_a - U_b (with the image velocity of b), wa, wb: the spins.
// The factors of a pair's lubrication terms that depend on the two radii
// only (the resistance functions of the gap aside): taken once per lattice
// step for the pairs a warp holds in registers, else in line.  Both give the
// same bits: the products and quotients are formed in the same order.
template <typename T>
struct LubK {
  T ra, rb;                                // the radii of a and b
  T xa, ya, yba, ybb, ycaa, ycbb, ycab;    // XA / inv, YA / lg, YB_a / lg, ... (radius factors)
  T sc, dl, xcdl, cinv;                    // 2 / (a_a + a_b), scaled roughness, xi_c + dl, 1 / (xi_c + dl)
};

template <typename T>
__device__ __forceinline__ void lub_factors(T ra, T rb, const PairConst<T>& pc, LubK<T>& k) {
  k.ra = ra;
  k.rb = rb;
  k.sc = (T)2 / (ra + rb);
  const T xc = k.sc * pc.lub_cut;
  k.dl = k.sc * pc.lub_delta;
  k.xcdl = xc + k.dl;
  k.cinv = (T)1 / (xc + k.dl);
  const T be = rb / ra, bj = ra / rb;
  const T pi = (T)3.14159265358979323846;
  const T e0 = pc.eta0;
  const T op = (T)1 + be, oq = (T)1 + bj;
  k.xa = e0 * (T)6 * pi * ra * ((T)2 * be * be / (op * op * op));
  k.ya = e0 * (T)6 * pi * ra * ((T)4 * be * ((T)2 + be + (T)2 * be * be) / ((T)15 * op * op * op));
  k.yba = e0 * (T)4 * pi * ra * ra * (be * ((T)4 + be) / ((T)5 * op * op));
  k.ybb = e0 * (T)4 * pi * rb * rb * (bj * ((T)4 + bj) / ((T)5 * oq * oq));
  k.ycaa = e0 * (T)8 * pi * ra * ra * ra * ((T)2 * be / ((T)5 * op));
  k.ycbb = e0 * (T)8 * pi * rb * rb * rb * ((T)2 * bj / ((T)5 * oq));
  k.ycab = e0 * (T)8 * pi * ra * ra * ra * (be * be / ((T)10 * op));
}

// lk: the pair's radius factors taken for the step, or NULL (in line).
template <typename T>
__device__ void pair_interact(const View& v, int a, int b, const T d[3], T h, const T uab[3], const T wa[3],
                              const T wb[3], const T spring[3], T dt, const PairConst<T>& pc, PairOut<T>& o,
                              bool want_s, const LubK<T>* lk) {
  const T* pl = reinterpret_cast<const T*>(v.plb);
  const T ra = lk ? lk->ra : pl[12 * a + 9], rb = lk ? lk->rb : pl[12 * b + 9];
  const T dist = sqrt(dot3(d, d));
  // FP32 compute takes its quotients and the lubrication logarithm from the
  // fast hardware forms (a few units in the last place; the FP64 path keeps
  // correctly rounded ones)
  T n[3];
  if constexpr (sizeof(T) == 4) {
    const float id = __fdividef(1.0f, dist);
    n[0] = d[0] * id; n[1] = d[1] * id; n[2] = d[2] * id;
  } else {
    n[0] = d[0] / dist; n[1] = d[1] / dist; n[2] = d[2] / dist;
  }
  for (int c = 0; c < 3; ++c) {
    o.Fa[c] = o.Ta[c] = o.Tb[c] = o.Fc[c] = o.Fr[c] = o.ht[c] = (T)0;
    o.d[c] = d[c];
  }
  o.fn = (T)0;
  o.touching = 0;
  for (int c = 0; c < 6; ++c) o.S[c] = (T)0;
  // ---- contact
  const T overlap = -h;   // (a_a + a_b) - |d|, from the accurate gap
  if (h < (T)0) {
    T ht[3] = {spring[0], spring[1], spring[2]};
    const T ws[3] = {ra * wa[0] + rb * wb[0], ra * wa[1] + rb * wb[1], ra * wa[2] + rb * wb[2]};
    T rot[3];
    cross3(ws, n, rot);
    const T vv[3] = {uab[0] + rot[0], uab[1] + rot[1], uab[2] + rot[2]};
    const T vn = dot3(vv, n);
    const T vt[3] = {vv[0] - vn * n[0], vv[1] - vn * n[1], vv[2] - vn * n[2]};
    const T kn = pc.kn, kt = pc.kt;
    const T fn = kn * overlap + pc.eta_n * vn;
    const T hn = dot3(ht, n);
    for (int c = 0; c < 3; ++c) ht[c] = ht[c] - hn * n[c] + vt[c] * dt;
    T ft[3] = {-kt * ht[0], -kt * ht[1], -kt * ht[2]};
    const T ftm = sqrt(dot3(ft, ft));
    const T cap = pc.mu * fabs(fn);
    if (ftm >= cap && ftm > (T)0) {
      if constexpr (sizeof(T) == 4) {
        const float sc = __fdividef(cap, ftm), ikt = __fdividef(1.0f, kt);
        for (int c = 0; c < 3; ++c) {
          ft[c] = ft[c] * sc;
          ht[c] = -ft[c] * ikt;
        }
      } else {
        for (int c = 0; c < 3; ++c) {
          ft[c] = cap * ft[c] / ftm;
          ht[c] = -ft[c] / kt;
        }
      }
    }
    T tq[3];
    cross3(n, ft, tq);
    for (int c = 0; c < 3; ++c) {
      o.Fc[c] = -fn * n[c] + ft[c];
      o.Fa[c] += o.Fc[c];
      o.Ta[c] += ra * tq[c];
      o.Tb[c] += rb * tq[c];
      o.ht[c] = ht[c];
    }
    o.fn = fn;
    o.touching = 1;
  }
  // ---- double-layer repulsion
  if (pc.rep && h < pc.debye10) {
    const T fr = pc.F0 * exp(-(h > (T)0 ? h : (T)0) / pc.debye);
    for (int c = 0; c < 3; ++c) {
      o.Fr[c] = -fr * n[c];
      o.Fa[c] += o.Fr[c];
    }
  }
  // ---- lubrication correction
  if (pc.lub && h < pc.lub_cut) {
    const T hh = h < (T)0 ? (T)0 : h;
    LubK<T> kl;
    if (!lk) lub_factors<T>(ra, rb, pc, kl);
    const LubK<T>& K = lk ? *lk : kl;
    const T xi = K.sc * hh, dl = K.dl;
    T inv, lg;
    if constexpr (sizeof(T) == 4) {
      const float ix = __fdividef(1.0f, xi + dl);
      inv = ix - K.cinv;
      lg = __logf(K.xcdl * ix);
    } else {
      inv = (T)1 / (xi + dl) - K.cinv;
      lg = log(K.xcdl / (xi + dl));
    }
    const T XA = K.xa * inv;
    const T YA = K.ya * lg;
    const T YBa = K.yba * lg;
    const T YBb = K.ybb * lg;
    const T YCaa = K.ycaa * lg;
    const T YCbb = K.ycbb * lg;
    const T YCab = K.ycab * lg;
    const T un = dot3(uab, n);
    T wan[3], wbn[3], nxu[3];
    cross3(wa, n, wan);
    cross3(wb, n, wbn);
    cross3(n, uab, nxu);
    const T wap = dot3(wa, n), wbp = dot3(wb, n);
    for (int c = 0; c < 3; ++c) {
      const T ut = uab[c] - un * n[c];
      o.Fa[c] += -XA * un * n[c] - YA * ut - YBa * wan[c] - YBb * wbn[c];
      const T wat = wa[c] - wap * n[c], wbt = wb[c] - wbp * n[c];
      o.Ta[c] += -YBa * nxu[c] - YCaa * wat - YCab * wbt;
      o.Tb[c] += -YBb * nxu[c] - YCbb * wbt - YCab * wat;
    }
    if (want_s) {
      const T be = rb / ra, bj = ra / rb;
      const T pi = (T)3.14159265358979323846;
      const T e0 = pc.eta0;
      const T op = (T)1 + be, oq = (T)1 + bj;
      // stresslets of both spheres (G and H blocks), each with its own radius
      // and beta = partner / own radius; the G terms are odd in (n, U_a - U_b)
      // and the H terms even in n, so both take n and uab:
      //   S = -[XG (n n - I/3)(n.U) + YG (n U + U n - 2 n n (n.U))
      //         + YH_a,self (Om_a x n) n + YH_a,other (Om_b x n) n + (b alike) + transposes]
      const T XG = e0 * (T)4 * pi * (ra * ra * ((T)3 * be * be / (op * op * op)) +
                                     rb * rb * ((T)3 * bj * bj / (oq * oq * oq))) * inv;
      const T YG = e0 * (T)4 * pi * (ra * ra * (be * ((T)4 - be + (T)7 * be * be) / ((T)10 * op * op * op)) +
                                     rb * rb * (bj * ((T)4 - bj + (T)7 * bj * bj) / ((T)10 * oq * oq * oq))) * lg;
      const T Hsa = ra * ra * ra * (be * ((T)2 - be) / ((T)10 * op * op));
      const T Hoa = ra * ra * ra * (be * be * ((T)1 + (T)7 * be) / ((T)20 * op * op));
      const T Hsb = rb * rb * rb * (bj * ((T)2 - bj) / ((T)10 * oq * oq));
      const T Hob = rb * rb * rb * (bj * bj * ((T)1 + (T)7 * bj) / ((T)20 * oq * oq));
      const T YHwa = e0 * (T)8 * pi * (Hsa + Hob) * lg;   // multiplies (Om_a x n) n + n (Om_a x n)
      const T YHwb = e0 * (T)8 * pi * (Hsb + Hoa) * lg;   // multiplies (Om_b x n) n + n (Om_b x n)
      const int ix[6] = {0, 1, 2, 0, 0, 1}, iy[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        const int x = ix[m], y = iy[m];
        const T g = XG * (n[x] * n[y] - (x == y ? (T)1 / (T)3 : (T)0)) * un +
                    YG * (n[x] * uab[y] + uab[x] * n[y] - (T)2 * n[x] * n[y] * un);
        const T hh = YHwa * (wan[x] * n[y] + n[x] * wan[y]) + YHwb * (wbn[x] * n[y] + n[x] * wbn[y]);
        o.S[m] = -(g + hh);
      }
    }
  }
}

template <typename T>
__device__ inline T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// State buffers of one sub-step.  Other warps write the read buffers during
// the launch (in earlier sub-steps), so they are never read through the
// non-coherent read-only path.
struct State {
  const double *R, *U, *W;   // read: positions and velocities at the sub-step start
  double *Rn, *Un, *Wn;      // write: after the sub-step
  const float* m;            // FP32 compute: mirror of the read buffer (R - Ro, U, W)
  float* mn;                 //  and of the write buffer
  void* pw;                  // compute-type copy written at the last sub-step: v.plb, or v.plb_next
                             // while the collide-stream still reads v.plb beside this kernel
};

// Particle i's entry of the compute-type copy at base (v.plb, or v.plb_next).
template <typename TC>
__device__ inline void write_plb(void* base, const View& v, int i, const double* R, const double* U,
                                 const double* W) {
  TC* pp = reinterpret_cast<TC*>(base) + 12 * i;
  for (int c = 0; c < 3; ++c) {
    pp[c] = (TC)R[c];
    pp[3 + c] = (TC)U[c];
    pp[6 + c] = (TC)W[c];
  }
  pp[9] = (TC)v.rad[i];
}

// Per-step constants of one particle, loaded once per lattice step when a
// warp holds a single particle for the whole step: the protocol offset and
// image velocity, the pair-force constants, and for its integration the held
// link plus covering force and torque and the inverse mass and inertia, in
// the compute type (the same conversions the per-sub-step path makes).
// The integration constants of particle i for one step, in the compute type:
// (T) F^h + (T) F^cov, (T) T^h + (T) T^cov, 1 / m, 1 / I.
template <typename T>
__device__ inline void integ_const(const View& v, int i, T (&k)[8]) {
  for (int a = 0; a < 3; ++a) {
    k[a] = (T)v.Fh[3 * i + a] + (T)v.Fcov[3 * i + a];
    k[3 + a] = (T)v.Th[3 * i + a] + (T)v.Tcov[3 * i + a];
  }
  k[6] = (T)v.inv_m[i];
  k[7] = (T)v.inv_I[i];
}

template <typename T>
struct StepConst {
  T delta, ule;
  double Ro[3];     // step-start centre (the FP32 mirror's origin)
  T k[8];           // integ_const
  double dt;        // 1 / n_sub
  PairConst<T> pc;
  float me[12];     // FP32 compute: the warp's own mirror (R - Ro, U, W at 0, 4, 8) of the current sub-step
};

template <typename T>
__device__ inline void load_step_const(const View& v, int i, StepConst<T>& c) {
  const Proto* pr = v.proto;
  c.delta = sel<T>(pr->delta, pr->delta_f);
  c.Ro[0] = v.Ro[3 * i]; c.Ro[1] = v.Ro[3 * i + 1]; c.Ro[2] = v.Ro[3 * i + 2];
  c.ule = sel<T>(pr->ule, pr->ule_f);
  integ_const<T>(v, i, c.k);
  c.dt = v.dt_sub;
  load_pair_const<T>(v, c.pc);
  // the mirror as the candidate search writes it for the first sub-step
  for (int q = 0; q < 3; ++q) {
    c.me[q] = 0.0f;
    c.me[4 + q] = (float)v.U[3 * i + q];
    c.me[8 + q] = (float)v.W[3 * i + q];
  }
}

// Semi-implicit Euler sub-step of particle i (Eq. 1) from the read state to
// the write state, with the pair force and torque (F, T); at the last sub-step
// the Lees-Edwards wrap of the centre, the speed check and the compute-type copy.
// Velocities are updated in precision T.  FP64 compute steps the FP64 state.
// FP32 compute steps the FP32 mirror (velocities, spin and the displacement
// since the step start, with no FP64 arithmetic) and at the last sub-step
// sets the FP64 centre to the step-start centre plus that displacement, so
// positions are FP64 at every lattice step.
template <typename T>
__device__ inline void integrate_one(const View& v, int i, const State& S, const T Fp[3], const T Tp[3],
                                     double dt, bool last, bool plb_double, const T* k, const double* Ro,
                                     float* me) {
  double R[3], U[3], W[3];
  const T im = k[6], iI = k[7], dtt = (T)dt;
  // A driven (wall) sphere keeps its velocity and spin whatever the forces.
  const bool driven = v.has_drv && v.drv[i];
  if constexpr (sizeof(T) == 4) {
    // this particle's mirror: the warp's copy in shared memory when it holds
    // the particle for the whole step (the same values as the read buffer)
    const float* m = me ? me : S.m + 12 * i;
    float Uf[3], Wf[3], df[3];
    for (int c = 0; c < 3; ++c) {
      Uf[c] = driven ? m[4 + c] : m[4 + c] + dtt * (k[c] + Fp[c]) * im;
      Wf[c] = driven ? m[8 + c] : m[8 + c] + dtt * (k[3 + c] + Tp[c]) * iI;
    }
    if (v.quasi2d && !driven) { Uf[2] = 0.0f; Wf[0] = 0.0f; Wf[1] = 0.0f; }
    for (int c = 0; c < 3; ++c) df[c] = m[c] + dtt * Uf[c];
    // the partners' FP32 view of this particle for the next sub-step
    float* mm = S.mn + 12 * i;
    for (int c = 0; c < 3; ++c) {
      mm[c] = df[c];
      mm[4 + c] = Uf[c];
      mm[8 + c] = Wf[c];
    }
    if (me)
      for (int c = 0; c < 3; ++c) {
        me[c] = df[c];
        me[4 + c] = Uf[c];
        me[8 + c] = Wf[c];
      }
    if (!last) return;
    // the FP64 state at the step's end (a driven sphere's velocity and spin
    // are its prescribed FP64 values, and it moves by exactly one step of them)
    for (int c = 0; c < 3; ++c) {
      U[c] = driven ? v.U[3 * i + c] : (double)Uf[c];
      W[c] = driven ? v.W[3 * i + c] : (double)Wf[c];
      R[c] = driven ? Ro[c] + U[c] : Ro[c] + (double)df[c];
    }
  } else {
    for (int c = 0; c < 3; ++c) {
      const T F = k[c] + Fp[c];
      const T Tq = k[3 + c] + Tp[c];
      U[c] = driven ? S.U[3 * i + c] : (double)((T)S.U[3 * i + c] + dtt * F * im);
      W[c] = driven ? S.W[3 * i + c] : (double)((T)S.W[3 * i + c] + dtt * Tq * iI);
    }
    if (v.quasi2d && !driven) { U[2] = 0.0; W[0] = 0.0; W[1] = 0.0; }
    for (int c = 0; c < 3; ++c) R[c] = S.R[3 * i + c] + dt * U[c];
  }
  if (last) {
    const Proto* pr = v.proto;
    const double du = driven ? 0.0 : pr->ule;   // a driven sphere's velocity is prescribed
    if (R[1] >= v.ny) { R[1] -= v.ny; R[0] -= pr->delta_n; U[0] -= du; }
    else if (R[1] < 0.0) { R[1] += v.ny; R[0] += pr->delta_n; U[0] += du; }
    if (R[0] < 0.0) R[0] += v.nx; else if (R[0] >= v.nx) R[0] -= v.nx;
    if (R[2] < 0.0) R[2] += v.nz; else if (R[2] >= v.nz) R[2] -= v.nz;
    const T sp2 = (T)(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    bool bad = !(sp2 < (T)0.25);
    // Centres stay finite and inside the box whatever the dynamics did: the
    // node-map kernels index the lattice from them.  x can still be one
    // period out after a Lees-Edwards crossing at the x boundary; anything
    // else out of range means the step was unstable.
    const int Ls[3] = {v.nx, v.ny, v.nz};
    for (int c = 0; c < 3; ++c) {
      if (R[c] >= 0.0 && R[c] < Ls[c]) continue;
      if (c != 0 || !isfinite(R[c])) bad = true;
      R[c] = isfinite(R[c]) ? R[c] - Ls[c] * floor(R[c] / Ls[c]) : 0.0;
      if (!(R[c] >= 0.0 && R[c] < Ls[c])) R[c] = 0.0;
    }
    if (bad) atomicOr(v.err, ERR_UNSTABLE);
    if (plb_double) write_plb<double>(S.pw, v, i, R, U, W);
    else write_plb<float>(S.pw, v, i, R, U, W);
  }
  for (int c = 0; c < 3; ++c) {
    S.Rn[3 * i + c] = R[c];
    S.Un[3 * i + c] = U[c];
    S.Wn[3 * i + c] = W[c];
  }
}

// Spring table of one step boundary: per particle a, its touching partners
// b > a and their tangential springs.  Step t reads table t & 1 and writes
// table (t + 1) & 1.
struct SpringTable {
  int* cnt;
  int* part;
  double* val;
};
__device__ inline SpringTable spring_table(const View& v, long long t) {
  return (t & 1) ? SpringTable{v.hcnt1, v.hpart1, v.hval1} : SpringTable{v.hcnt0, v.hpart0, v.hval0};
}

// Candidate partners of particle i for one lattice step, collected by one
// warp at the step start: every particle whose centre lies within
// a_i + a_j + (interaction range) + 1 (particles move less than 0.5 per step,
// so no pair that interacts during the step is missed).  Entry c of the
// particle's scratch row holds the partner index and the pair's tangential
// spring, initialised from the spring table.  Returns the count (all lanes).
template <typename T>
__device__ int collect_pairs(const View& v, int i, const SpringTable& old) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const double* R = v.R;
  const double Rx = R[3 * i], Ry = R[3 * i + 1], Rz = R[3 * i + 2];
  const double ai = v.rad[i];
  const double delta = v.proto->delta;
  const double skin = v.hrange + 1.0;
  int* pj = v.pj + (long long)i * PAIR_SLOTS;
  T* ph = reinterpret_cast<T*>(v.ph) + 3LL * i * PAIR_SLOTS;   // springs in the compute type
  int base = 0;
  auto consider = [&](int j, bool valid) {
    bool take = false;
    if (valid && j != i) {
      double dx = R[3 * j] - Rx, dy = R[3 * j + 1] - Ry, dz = R[3 * j + 2] - Rz;
      le_image<double>(dx, dy, dz, delta, v.nx, v.ny, v.nz, v.inv_nx_d, v.inv_ny_d, v.inv_nz_d);
      const double lim = ai + v.rad[j] + skin;
      take = dx * dx + dy * dy + dz * dz < lim * lim;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (take) {
      const int c = base + __popc(bal & lt);
      if (c < PAIR_SLOTS) {
        pj[c] = j;
        // the spring of the canonical pair lives in the table of a = min(i, j)
        const int a = i < j ? i : j, b = i < j ? j : i;
        double h0 = 0.0, h1 = 0.0, h2 = 0.0;
        const int m = old.cnt[a];
        for (int s = 0; s < m; ++s)
          if (old.part[a * v.K + s] == b) {
            h0 = old.val[3 * (a * v.K + s)]; h1 = old.val[3 * (a * v.K + s) + 1]; h2 = old.val[3 * (a * v.K + s) + 2];
            break;
          }
        ph[3 * c] = (T)h0; ph[3 * c + 1] = (T)h1; ph[3 * c + 2] = (T)h2;
      }
    }
    base += __popc(bal);
  };
  if (v.brute) {
    // every particle, from the compute-type copy (R, radius); a 0.01 margin
    // covers its rounding, so the set still holds every interacting pair
    const T* pl = reinterpret_cast<const T*>(v.plb);
    const T px = pl[12 * i], py = pl[12 * i + 1], pz = pl[12 * i + 2], pa = pl[12 * i + 9];
    const T dl = (T)delta, sk = (T)(skin + 0.01);
    int rbase = 0;
    // 8 candidates per lane and round: their loads are issued together
    constexpr int CU = 8;
    for (int j0 = 0; j0 < v.n; j0 += 32 * CU) {
      T cx[CU], cy[CU], cz[CU], cr[CU];
#pragma unroll
      for (int u = 0; u < CU; ++u) {
        const int j = j0 + 32 * u + lane;
        const bool ok = j < v.n;
        cx[u] = ok ? pl[12 * j] : (T)0;
        cy[u] = ok ? pl[12 * j + 1] : (T)0;
        cz[u] = ok ? pl[12 * j + 2] : (T)0;
        cr[u] = ok ? pl[12 * j + 9] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < CU; ++u) {
        const int j = j0 + 32 * u + lane;
        bool take = false;
        if (j < v.n && j != i) {
          T dx = cx[u] - px, dy = cy[u] - py, dz = cz[u] - pz;
          le_image_v<T>(v, dx, dy, dz, dl);
          const T lim = pa + cr[u] + sk;
          take = dx * dx + dy * dy + dz * dz < lim * lim;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (take) {
          const int c = rbase + __popc(bal & lt);
          if (c < PAIR_SLOTS) pj[c] = j;
        }
        rbase += __popc(bal);
      }
    }
    // springs of the candidates (lanes over the list)
    const int m = rbase < PAIR_SLOTS ? rbase : PAIR_SLOTS;
    __syncwarp();
    for (int c = lane; c < m; c += 32) {
      const int j = pj[c];
      const int a = i < j ? i : j, b = i < j ? j : i;
      // all slots of a's row at once (the table has HSLOTS_DEV slots per particle)
      const int mm = old.cnt[a];
      int hit = -1;
#pragma unroll
      for (int s = 0; s < HSLOTS_DEV; ++s) {
        const int pb = old.part[a * HSLOTS_DEV + s];
        if (s < mm && pb == b && hit < 0) hit = s;
      }
      double h0 = 0.0, h1 = 0.0, h2 = 0.0;
      if (hit >= 0) {
        const double* hv = old.val + 3 * (a * HSLOTS_DEV + hit);
        h0 = hv[0]; h1 = hv[1]; h2 = hv[2];
      }
      ph[3 * c] = (T)h0; ph[3 * c + 1] = (T)h1; ph[3 * c + 2] = (T)h2;
    }
    base = rbase;
  } else {
    // lane l < 27 owns neighbour cell l of i's cell at the step start; the
    // lanes walk their cells' entries in lockstep rounds
    int s0 = 0, cnt = 0;
    if (lane < 27) {
      const int dyc = lane / 9 - 1, dxc = (lane / 3) % 3 - 1, dzc = lane % 3 - 1;
      const int zlo = v.ncz >= 3 ? -1 : 0, zhi = v.ncz >= 2 ? 1 : 0;
      if (dzc >= zlo && dzc <= zhi) {
        const int* pc = v.pcx + 8 * i;
        int yc = pc[1] + dyc, cxs = pc[0];
        if (yc < 0) { yc += v.ncy; cxs = pc[3]; }
        else if (yc >= v.ncy) { yc -= v.ncy; cxs = pc[4]; }
        const int xc = wrapi(cxs + dxc, v.ncx);
        const int zc = wrapi(pc[2] + dzc, v.ncz);
        const int c = xc + v.ncx * (yc + v.ncy * zc);
        s0 = v.cell_start[c];
        cnt = v.cell_start[c + 1] - s0;
      }
    }
    const int rounds = __reduce_max_sync(0xffffffffu, cnt);
    for (int r = 0; r < rounds; ++r) consider(r < cnt ? v.cell_ids[s0 + r] : -1, r < cnt);
  }
  if (base > PAIR_SLOTS && lane == 0) atomicOr(v.err, ERR_PAIRS);
  const int m = base < PAIR_SLOTS ? base : PAIR_SLOTS;
  if constexpr (sizeof(T) == 4) {
    // FP32 compute: each candidate's step constants in the canonical
    // orientation (a < b), so that both partners hold the same bits
    __syncwarp();
    for (int c = lane; c < m; c += 32) {
      const int j = pj[c];
      const int a = i < j ? i : j, b = i < j ? j : i;
      double dx = R[3 * b] - R[3 * a], dy = R[3 * b + 1] - R[3 * a + 1], dz = R[3 * b + 2] - R[3 * a + 2];
      const int k = le_image<double>(dx, dy, dz, delta, v.nx, v.ny, v.nz, v.inv_nx_d, v.inv_ny_d, v.inv_nz_d);
      const double rs = v.rad[a] + v.rad[b];
      v.pd[(long long)i * PAIR_SLOTS + c] =
          make_float4((float)dx, (float)dy, (float)dz, (float)(dx * dx + dy * dy + dz * dz - rs * rs));
      v.pk[(long long)i * PAIR_SLOTS + c] = (signed char)k;
    }
  }
  return m;
}

// Pair forces on particle i for one sub-step, computed by one warp: lane l
// takes candidates l and l + 32, evaluates each pair in its canonical
// orientation (a = min, b = max; both partners compute bitwise the same
// result, so no atomics) and carries the pair's spring in the scratch row.
// Sums are reduced across the warp; lane 0 integrates.  At the box's last
// sub-step the particle's touching pairs with larger partners go to the
// spring table of the next step.
// A lane's candidates (slots lane and lane + 32) and their springs, kept in
// registers across the sub-steps when a warp holds one particle for the step.
template <typename T>
struct PairRegs {
  int j[PAIR_SLOTS / 32];
  T h[PAIR_SLOTS / 32][3];   // (springs are exact in T: each is a T result)
  float4 D[PAIR_SLOTS / 32];   // FP32 compute: the pair's step constants (D, c0)
  int k[PAIR_SLOTS / 32];      //  and image index
};

// Sum over the LANES lanes of a lane group (a warp or a half-warp).
template <int LANES, typename T>
__device__ __forceinline__ T group_sum(T x) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// One sub-step of particle i, computed by a group of LANES lanes (the whole
// warp, or one half when a warp takes two particles; every lane of the warp
// calls this together).  valid = false: the group has no particle this time
// and only takes part in the shuffles.
template <typename T, int LANES>
__device__ __forceinline__ void pairs_of(const View& v, int i, int npairs, bool valid, const State& S, T dt,
                                         int sample, bool last, const SpringTable& next,
                                         StepConst<T>* sc, PairRegs<T>* rg, const LubK<T>* lkw, bool fresh) {
  constexpr int NS = PAIR_SLOTS / LANES;   // candidate slots per lane
  const int lane = threadIdx.x & (LANES - 1);
  const int grp_shift = (threadIdx.x & 31) & ~(LANES - 1);   // first lane of the group
  if (!valid) npairs = 0;
  const Proto* pr = v.proto;
  const T delta = sc ? sc->delta : sel<T>(pr->delta, pr->delta_f);
  const T ule = sc ? sc->ule : sel<T>(pr->ule, pr->ule_f);
  PairConst<T> pcl;
  if (!sc) load_pair_const<T>(v, pcl);
  const PairConst<T>& pc = sc ? sc->pc : pcl;
  T F[3] = {0, 0, 0}, Tq[3] = {0, 0, 0};
  T cv[9], rv[9], lv[6];
  for (int c = 0; c < 9; ++c) { cv[c] = (T)0; rv[c] = (T)0; }
  for (int c = 0; c < 6; ++c) lv[c] = (T)0;
  int ncont = 0;
  const double pi = 3.14159265358979323846;
  const double dth = pi / v.nbins;
  int* pj = v.pj + (long long)i * PAIR_SLOTS;
  T* ph = reinterpret_cast<T*>(v.ph) + 3LL * i * PAIR_SLOTS;
  bool keep[NS] = {};   // touching pair with i = a after this sub-step
#pragma unroll
  for (int slot = 0; slot < NS; ++slot) {
    const int c = lane + LANES * slot;
    if (c >= npairs) continue;
    const int j = rg ? rg->j[slot] : pj[c];
    const int a = i < j ? i : j, b = i < j ? j : i;
    T d[3], h, uab[3], wa[3], wb[3];
    bool touching = false, inr;
    if constexpr (sizeof(T) == 8) {
      int k;
      inr = pair_geometry<T>(v, S.R, a, b, delta, pc, d, k, h);
      if (inr) {
        for (int x = 0; x < 3; ++x) {
          uab[x] = S.U[3 * a + x] - S.U[3 * b + x];
          wa[x] = S.W[3 * a + x];
          wb[x] = S.W[3 * b + x];
        }
        uab[0] -= (T)k * ule;
      }
    } else {
      // d = D + (e_b - e_a) with e the FP32 displacements since the step
      // start; |d|^2 - (a_a + a_b)^2 = c0 + (2 D + e) . e, so the gap keeps
      // the accuracy of the step's FP64 constants (no cancellation in FP32)
      const float4 D = rg ? rg->D[slot] : v.pd[(long long)i * PAIR_SLOTS + c];
      const int k = rg ? rg->k[slot] : (int)v.pk[(long long)i * PAIR_SLOTS + c];
      // both mirrors, 16-byte aligned rows of 12 (d, U, W and pads), all six
      // loads issued together
      float4 da, db, ua4, ub4, wa4, wb4;
      if (fresh) {
        // the first sub-step: the mirrors' step-start values (no
        // displacement, U and Omega of the FP64 state), read from the state
        // itself rather than from the mirrors the candidate search writes
        da = db = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        ua4 = make_float4((float)v.U[3 * a], (float)v.U[3 * a + 1], (float)v.U[3 * a + 2], 0.0f);
        ub4 = make_float4((float)v.U[3 * b], (float)v.U[3 * b + 1], (float)v.U[3 * b + 2], 0.0f);
        wa4 = make_float4((float)v.W[3 * a], (float)v.W[3 * a + 1], (float)v.W[3 * a + 2], 0.0f);
        wb4 = make_float4((float)v.W[3 * b], (float)v.W[3 * b + 1], (float)v.W[3 * b + 2], 0.0f);
      } else {
        const float4* qa = reinterpret_cast<const float4*>(S.m + 12 * a);
        const float4* qb = reinterpret_cast<const float4*>(S.m + 12 * b);
        da = qa[0]; db = qb[0]; ua4 = qa[1]; ub4 = qb[1]; wa4 = qa[2]; wb4 = qb[2];
      }
      const float ex = db.x - da.x, ey = db.y - da.y, ez = db.z - da.z;
      const float num = D.w + ((2.0f * D.x + ex) * ex + ((2.0f * D.y + ey) * ey + (2.0f * D.z + ez) * ez));
      const float* pl = reinterpret_cast<const float*>(v.plb);
      const float rsum = lkw ? lkw[c].ra + lkw[c].rb : pl[12 * a + 9] + pl[12 * b + 9];
      inr = num < pc.hrange * (2.0f * rsum + pc.hrange) + 1e-5f;
      if (inr) {
        d[0] = D.x + ex; d[1] = D.y + ey; d[2] = D.z + ez;
        h = __fdividef(num, sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) + rsum);
        inr = (h < pc.hrange) || (h < 0.0f);
        uab[0] = ua4.x - ub4.x; uab[1] = ua4.y - ub4.y; uab[2] = ua4.z - ub4.z;
        wa[0] = wa4.x; wa[1] = wa4.y; wa[2] = wa4.z;
        wb[0] = wb4.x; wb[1] = wb4.y; wb[2] = wb4.z;
        uab[0] -= (float)k * ule;
      }
    }
    if (inr) {
      T spring[3];
      for (int x = 0; x < 3; ++x) spring[x] = rg ? rg->h[slot][x] : ph[3 * c + x];
      PairOut<T> o;
      pair_interact<T>(v, a, b, d, h, uab, wa, wb, spring, dt, pc, o, sample && i == a, lkw ? lkw + c : nullptr);
      touching = o.touching != 0;
      for (int x = 0; x < 3; ++x) {
        if (rg) rg->h[slot][x] = touching ? o.ht[x] : (T)0;
        else ph[3 * c + x] = touching ? o.ht[x] : (T)0;
      }
      if (i == a) {
        for (int x = 0; x < 3; ++x) { F[x] += o.Fa[x]; Tq[x] += o.Ta[x]; }
        keep[slot] = touching;
        if (sample) {
          const T r[3] = {-o.d[0], -o.d[1], -o.d[2]};
          if (touching) {
            for (int x = 0; x < 3; ++x)
              for (int y = 0; y < 3; ++y) cv[3 * x + y] += (T)0.5 * (r[x] * o.Fc[y] + r[y] * o.Fc[x]);
            // contact angle theta in [0, pi) and the tangential direction
            // t = (-sin theta, cos theta) of the unfolded angle (Eq. 26, 27);
            // the tangential force is counted positive when it turns the
            // spheres counter-clockwise, -(F_a . t) (a's contact point lies
            // at -a n from its centre)
            int bin;
            double ftan;
            if constexpr (sizeof(T) == 8) {
              double th = atan2((double)r[1], (double)r[0]);
              const double tx = -sin(th), ty = cos(th);
              if (th < 0.0) th += pi;
              if (th >= pi) th -= pi;
              bin = (int)floor(th / dth);
              ftan = -((double)o.Fc[0] * tx + (double)o.Fc[1] * ty);
            } else {
              // FP32 angles: the same bins but at the edges; the direction
              // straight from r (no trigonometry)
              const float pf = 3.14159265358979323846f;
              float th = atan2f((float)r[1], (float)r[0]);
              const float rr = sqrtf((float)r[0] * (float)r[0] + (float)r[1] * (float)r[1]);
              const float tx = rr > 0.0f ? -(float)r[1] / rr : 0.0f, ty = rr > 0.0f ? (float)r[0] / rr : 1.0f;
              if (th < 0.0f) th += pf;
              if (th >= pf) th -= pf;
              bin = (int)floorf(th * ((float)v.nbins / pf));
              ftan = -(double)((float)o.Fc[0] * tx + (float)o.Fc[1] * ty);
            }
            if (bin >= v.nbins) bin = v.nbins - 1;
            if (bin < 0) bin = 0;
            atomicAdd(v.hist + 3 * bin, 1.0);
            atomicAdd(v.hist + 3 * bin + 1, (double)o.fn);
            atomicAdd(v.hist + 3 * bin + 2, ftan);
            ++ncont;
          }
          if (v.F0 > 0.0)
            for (int x = 0; x < 3; ++x)
              for (int y = 0; y < 3; ++y) rv[3 * x + y] += (T)0.5 * (r[x] * o.Fr[y] + r[y] * o.Fr[x]);
          for (int c = 0; c < 6; ++c) lv[c] += o.S[c];
        }
      } else {
        for (int x = 0; x < 3; ++x) { F[x] -= o.Fa[x]; Tq[x] += o.Tb[x]; }
      }
    } else if (rg) {
      rg->h[slot][0] = (T)0; rg->h[slot][1] = (T)0; rg->h[slot][2] = (T)0;
    } else {
      ph[3 * c] = (T)0; ph[3 * c + 1] = (T)0; ph[3 * c + 2] = (T)0;
    }
  }
  for (int c = 0; c < 3; ++c) { F[c] = group_sum<LANES>(F[c]); Tq[c] = group_sum<LANES>(Tq[c]); }
  if (sample) {
    for (int c = 0; c < 9; ++c) { cv[c] = group_sum<LANES>(cv[c]); rv[c] = group_sum<LANES>(rv[c]); }
    if (pc.lub)
      for (int c = 0; c < 6; ++c) lv[c] = group_sum<LANES>(lv[c]);
    ncont = group_sum<LANES>(ncont);
  }
  if (last) {
    // touching pairs (i, b > i) in candidate order -> next step's table
    int base = 0;
#pragma unroll
    for (int slot = 0; slot < NS; ++slot) {
      const unsigned all = __ballot_sync(0xffffffffu, keep[slot]);
      const unsigned bal = LANES == 32 ? all : (all >> grp_shift) & ((1u << (LANES & 31)) - 1u);
      if (keep[slot]) {
        const int m = base + __popc(bal & ((1u << lane) - 1u));
        const int c = lane + LANES * slot;
        if (m < v.K) {
          next.part[i * v.K + m] = rg ? rg->j[slot] : pj[c];
          for (int x = 0; x < 3; ++x)
            next.val[3 * (i * v.K + m) + x] = (double)(rg ? rg->h[slot][x] : ph[3 * c + x]);
        }
      }
      base += __popc(bal);
    }
    if (lane == 0 && valid) {
      next.cnt[i] = base < v.K ? base : v.K;
      if (base > v.K) atomicOr(v.err, ERR_PAIRS);
    }
  }
  __syncwarp();
  if (lane == 0 && valid) {
    integrate_one<T>(v, i, S, F, Tq, sc ? sc->dt : v.dt_sub, last, sizeof(T) == 8,
                     sc ? sc->k : reinterpret_cast<const T*>(v.pconst) + 8 * i, sc ? sc->Ro : v.Ro + 3 * i,
                     sc ? sc->me : nullptr);
    if (sample) {
      for (int c = 0; c < 9; ++c) {
        atomicAdd(acc_rep(v, i) + 15 + c, (double)cv[c]);
        if (v.F0 > 0.0) atomicAdd(acc_rep(v, i) + 25 + c, (double)rv[c]);
      }
      if (ncont) atomicAdd(acc_rep(v, i) + 24, (double)ncont);
      if (pc.lub)
        for (int c = 0; c < 6; ++c) atomicAdd(acc_rep(v, i) + 34 + c, (double)lv[c]);
    }
  }
  __syncwarp();
}

template <typename TC>
__device__ inline void write_plb(const View& v, int i) {
  write_plb<TC>(v.plb, v, i, v.R + 3 * i, v.U + 3 * i, v.W + 3 * i);
}

// All particle sub-steps of one lattice step, for every box, in one
// cooperative launch.  Per sub-step each warp computes one particle's pair
// forces from the state buffer read in that sub-step and its lane 0
// integrates the particle into the other buffer, so one grid-wide barrier per
// sub-step suffices; boxes with fewer sub-steps idle in the later rounds.  The
// final state ends in the canonical buffer (R, U, W).
// Warps (particles in flight) per block of the cooperative particle kernel:
// six warps at the FP32 path's 168 registers take 32 256 of an SM's 65 536,
// so one block fits beside one 256-thread collide-stream block of 128
// registers when the two kernels overlap.
#ifndef DEM_WARPS
#define DEM_WARPS 6
#endif

// End of the lattice step for every box of the batch, once every sub-step's
// forces and virials are in: one block per box (a block takes several boxes
// when the grid is smaller than the batch).  Saves the separate finalisation
// launch whenever particles move -- unless the collide-stream runs beside
// this kernel (B.dem_fin = 0): its viscous sums are then still coming and
// the finalisation is a launch of its own after both.
__device__ __forceinline__ void finalize_boxes(const Batch& B, cooperative_groups::grid_group& grid) {
  if (!B.dem_fin) return;
  grid.sync();
  for (int b = blockIdx.x; b < B.nbox; b += gridDim.x) {
    finalize_box(B.views[b]);
    __syncthreads();   // the block's shared totals are reused by its next box
  }
}

// SINGLE: the form for at most one particle per warp (the host launches it
// only when the grid's warps cover every particle), the other for more;
// two kernels keep each one's code small.
template <typename T, bool SINGLE>
__global__ void __launch_bounds__(32 * DEM_WARPS, sizeof(T) == 4 ? 2 : 1) k_dem_step(Batch B) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int wib = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * DEM_WARPS + wib, nwarps = gridDim.x * DEM_WARPS;
  const int ntot = B.part_off[B.nbox];
  // candidate partners of every moving particle at the step start
  int my_np = 0;   // candidate count of this warp's last particle (all lanes)
  for (int g = gwarp; g < ntot; g += nwarps) {
    const int bx = box_of(B.part_off, B.nbox, g);
    const View& v = B.views[bx];
    if (!v.move) continue;
    const int i = g - B.part_off[bx];
    const int np = collect_pairs<T>(v, i, spring_table(v, v.proto->t));
    if ((threadIdx.x & 31) == 0) {
      v.pcnt[i] = np;
      T k[8];
      integ_const<T>(v, i, k);
      T* dst = reinterpret_cast<T*>(v.pconst) + 8 * i;
      for (int c = 0; c < 8; ++c) dst[c] = k[c];
      if constexpr (sizeof(T) == 4) {
        // the step's origin and both buffers' FP32 mirrors (zero displacement)
        for (int c = 0; c < 3; ++c) {
          v.Ro[3 * i + c] = v.R[3 * i + c];
          for (int q = 0; q < 2; ++q) {
            float* mm = v.m32[q] + 12 * i;
            mm[c] = 0.0f;
            mm[4 + c] = (float)v.U[3 * i + c];
            mm[8 + c] = (float)v.W[3 * i + c];
          }
        }
      }
    }
    my_np = np;
  }
  bool any_odd = false;
  for (int b = 0; b < B.nbox; ++b) {
    const View& v = B.views[b];
    if (v.move && v.n > 0 && (v.nsub & 1)) any_odd = true;
  }
  if (any_odd) {
    // odd sub-step count: the first sub-step reads a copy in the second
    // buffer (and writes the canonical one, so every warp's candidate search
    // above must be done first)
    grid.sync();
    const int gthr = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    for (int g = gthr; g < ntot; g += nthr) {
      const int bx = box_of(B.part_off, B.nbox, g);
      const View& v = B.views[bx];
      if (!v.move || !(v.nsub & 1)) continue;
      const int i = g - B.part_off[bx];
      for (int c = 0; c < 3; ++c) {
        v.R2[3 * i + c] = v.R[3 * i + c]; v.U2[3 * i + c] = v.U[3 * i + c]; v.W2[3 * i + c] = v.W[3 * i + c];
      }
    }
    grid.sync();
  }
  if constexpr (SINGLE) {
    // at most one particle per warp: its per-step constants stay in registers.
    // A warp takes the same particle as in the candidate search above, and
    // the first sub-step reads its partners' step-start values from the
    // state rather than from the mirrors that search writes, so no barrier
    // comes between the two.
    const int g = gwarp;
    bool has = false;
    int bx = 0, i = 0, nsub = 0;
    if (g < ntot) {
      bx = box_of(B.part_off, B.nbox, g);
      i = g - B.part_off[bx];
      has = B.views[bx].move != 0;
    }
    const View& v = B.views[bx];
    __shared__ StepConst<T> s_sc[DEM_WARPS];
    StepConst<T>& sc = s_sc[wib];
    // FP32 compute: each warp's pairs' radius factors for the step
    __shared__ LubK<T> s_lk[sizeof(T) == 4 ? DEM_WARPS : 1][sizeof(T) == 4 ? PAIR_SLOTS : 1];
    SpringTable nxt{};
    State toA{}, toB{};
    if (has) {
      nsub = v.nsub;
      if ((threadIdx.x & 31) == 0) load_step_const<T>(v, i, sc);
      __syncwarp();
      nxt = spring_table(v, v.proto->t + 1);
      void* pw = B.dem_fin ? v.plb : v.plb_next;
      toA = State{v.R2, v.U2, v.W2, v.R, v.U, v.W, v.m32[1], v.m32[0], pw};
      toB = State{v.R, v.U, v.W, v.R2, v.U2, v.W2, v.m32[0], v.m32[1], pw};
    }
    const T dt = has ? (T)v.dt_sub : (T)0;
    PairRegs<T> rg;
#pragma unroll
    for (int slot = 0; slot < PAIR_SLOTS / 32; ++slot) {
      const int c = (threadIdx.x & 31) + 32 * slot;
      rg.j[slot] = 0;
      rg.h[slot][0] = rg.h[slot][1] = rg.h[slot][2] = (T)0;
      rg.D[slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      rg.k[slot] = 0;
      if (has && c < my_np) {
        const T* ph = reinterpret_cast<const T*>(v.ph) + 3LL * i * PAIR_SLOTS;
        rg.j[slot] = v.pj[(long long)i * PAIR_SLOTS + c];
        rg.h[slot][0] = ph[3 * c]; rg.h[slot][1] = ph[3 * c + 1]; rg.h[slot][2] = ph[3 * c + 2];
        if constexpr (sizeof(T) == 4) {
          rg.D[slot] = v.pd[(long long)i * PAIR_SLOTS + c];
          rg.k[slot] = v.pk[(long long)i * PAIR_SLOTS + c];
          // the pair's radius factors for the step (the lane that takes the slot)
          const int j = rg.j[slot], a = i < j ? i : j, b = i < j ? j : i;
          const float* pl = reinterpret_cast<const float*>(v.plb);
          lub_factors<float>(pl[12 * a + 9], pl[12 * b + 9], sc.pc, s_lk[wib][c]);
        }
      }
    }
    for (int sub = 0; sub < B.max_nsub; ++sub) {
      if (has && sub < nsub) {
        // sub-step s reads A when (nsub - s) is even, so the last write lands in A
        const State& S = ((nsub - sub) & 1) ? toA : toB;
        pairs_of<T, 32>(v, i, my_np, true, S, dt, sub == 0, sub == nsub - 1, nxt, &sc, &rg,
                        sizeof(T) == 4 ? s_lk[wib] : nullptr, sub == 0);
      }
      if (sub + 1 < B.max_nsub) grid.sync();
    }
    finalize_boxes(B, grid);
    return;
  }
  // Many particles per warp: two at a time, one per half-warp (16 lanes and
  // four candidate slots each), so that two latency chains run per warp.  The
  // halves take other particles than the candidate search did: one grid
  // barrier first.
  if (!any_odd) grid.sync();
  for (int sub = 0; sub < B.max_nsub; ++sub) {
    for (int gp = gwarp; 2 * gp < ntot; gp += nwarps) {
      const int g = 2 * gp + ((threadIdx.x >> 4) & 1);
      int bx = 0, i = 0;
      bool valid = g < ntot;
      if (valid) {
        bx = box_of(B.part_off, B.nbox, g);
        i = g - B.part_off[bx];
      }
      const View& v = B.views[bx];
      const int nsub = v.nsub;
      valid = valid && v.move && sub < nsub;
      // sub-step s reads A when (nsub - s) is even, so the last write lands in A
      void* pw = B.dem_fin ? v.plb : v.plb_next;
      const State toA{v.R2, v.U2, v.W2, v.R, v.U, v.W, v.m32[1], v.m32[0], pw};
      const State toB{v.R, v.U, v.W, v.R2, v.U2, v.W2, v.m32[0], v.m32[1], pw};
      const State& S = ((nsub - sub) & 1) ? toA : toB;
      pairs_of<T, 16>(v, i, valid ? v.pcnt[i] : 0, valid, S, (T)v.dt_sub, sub == 0, sub == nsub - 1,
                      spring_table(v, v.proto->t + 1), nullptr, nullptr, nullptr, false);
    }
    if (sub + 1 < B.max_nsub) grid.sync();
  }
  finalize_boxes(B, grid);
}

__global__ void k_write_plb(View v, int plb_double) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  if (plb_double) write_plb<double>(v, i);
  else write_plb<float>(v, i);
}

}  // namespace susp_dev

using namespace susp_dev;

void launch_write_plb(const View& v, int plb_double, cudaStream_t s) {
  if (v.n == 0) return;
  k_write_plb<<<(v.n + 127) / 128, 128, 0, s>>>(v, plb_double);
}

// Co-resident block count of the cooperative particle kernel for n particles.
int dem_grid_blocks(int plb_double, int n) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // both forms must fit: the one launched depends on the grid this returns
  int p1 = 0, p2 = 0;
  if (plb_double) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_dem_step<double, true>, 32 * DEM_WARPS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_dem_step<double, false>, 32 * DEM_WARPS, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_dem_step<float, true>, 32 * DEM_WARPS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_dem_step<float, false>, 32 * DEM_WARPS, 0);
  }
  per = p1 < p2 ? p1 : p2;
  if (per < 1) per = 1;
  if (sms < 1) sms = 1;
  const int want = (n + DEM_WARPS - 1) / DEM_WARPS;
  const int cap = sms * per;
  return want < cap ? (want > 0 ? want : 1) : cap;
}

// All particle sub-steps of one lattice step for every box of the batch: the
// cell lists (valid for every sub-step: the cells are at least one lattice
// unit wider than the interaction range and a particle moves less than 0.5
// per step), then one cooperative launch for the pair forces and integrations.
cudaError_t launch_dem_step(const Batch& B, int nparts, int ncells, int plb_double, int grid, cudaStream_t s) {
  if (nparts == 0) return cudaSuccess;
  const int nb = (nparts + 127) / 128;
  if (ncells > 0) {
    k_cell_count<<<nb, 128, 0, s>>>(B);
    k_cell_scan<<<B.nbox, 1024, 0, s>>>(B);
    k_cell_fill<<<nb, 128, 0, s>>>(B);
    k_cell_sort<<<(ncells + 127) / 128, 128, 0, s>>>(B);
  }
  Batch bb = B;
  void* args[] = {&bb};
  const bool single = nparts <= grid * DEM_WARPS;   // one particle per warp at most
  const void* fn = plb_double ? (single ? (const void*)k_dem_step<double, true> : (const void*)k_dem_step<double, false>)
                              : (single ? (const void*)k_dem_step<float, true> : (const void*)k_dem_step<float, false>);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(32 * DEM_WARPS), args, 0, s);
}
