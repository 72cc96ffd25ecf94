// susp_dev.cuh — device-side definitions shared by the CUDA translation units
// of the sheared-suspension step (lattice, storage traits, state views).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace susp_dev {

// ---------------------------------------------------------------- D3Q19
// Velocity set of Appendix A with weights C^q = 1/3, 1/18, 1/36; the order is
// the one documented in include/susp.h.
struct D3Q19 {
  static constexpr int Q = 19;
  // components packed as (c + 1) in two bits per direction:
  //   cx = 0 1 -1 0 0 0 0 1 -1 1 -1 1 -1 1 -1 0 0 0 0
  //   cy = 0 0 0 1 -1 0 0 1 -1 -1 1 0 0 0 0 1 -1 1 -1
  //   cz = 0 0 0 0 0 1 -1 0 0 0 0 1 -1 -1 1 1 -1 -1 1
  // (directions 0-15 in the first 32-bit word, 16-18 in the second)
  __host__ __device__ static constexpr int unpack(unsigned a, unsigned b, int q) {
    return (int)(((q < 16 ? a >> (2 * q) : b >> (2 * (q - 16)))) & 3u) - 1;
  }
  __host__ __device__ static constexpr int cx(int q) { return unpack(0x48889549u, 0x15u, q); }
  __host__ __device__ static constexpr int cy(int q) { return unpack(0x95609495u, 0x8u, q); }
  __host__ __device__ static constexpr int cz(int q) { return unpack(0xa0954955u, 0x20u, q); }
  // opposite direction: pairs (1,2) (3,4) ... (17,18)
  __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

// ------------------------------------------------------------ storage traits
// P = 0 FP64, 1 FP32, 2 FP16 deviation, 3 BF16 deviation from C^q rho0.
template <int P> struct Store;
template <> struct Store<0> {
  using T = double; using C = double;
  template <typename I> __device__ static C load(const T* f, I i, C, C) { return f[i]; }
  __device__ static T enc(C v, C, C) { return v; }
};
template <> struct Store<1> {
  using T = float; using C = float;
  template <typename I> __device__ static C load(const T* f, I i, C, C) { return __ldg(f + i); }
  __device__ static T enc(C v, C, C) { return v; }
  // value of element e from the aligned 32-bit word that holds it
  __device__ static C from_word(uint32_t w, uint32_t, C, C) { return __uint_as_float(w); }
};
template <> struct Store<2> {
  using T = __half; using C = float;
  // value = base + stored / scale
  template <typename I> __device__ static C load(const T* f, I i, C base, C inv_scale) {
    return base + __half2float(f[i]) * inv_scale;
  }
  __device__ static T enc(C v, C base, C scale) { return __float2half_rn((v - base) * scale); }
};
template <> struct Store<3> {
  using T = __nv_bfloat16; using C = float;
  template <typename I> __device__ static C load(const T* f, I i, C base, C inv_scale) {
    return base + __bfloat162float(f[i]) * inv_scale;
  }
  __device__ static T enc(C v, C base, C scale) { return __float2bfloat16_rn((v - base) * scale); }
};

// ------------------------------------------------------------ protocol state
// Lees-Edwards state of the current step t (transition t -> t+1): offset
// Delta_t (compensated sum), image velocity U_t = Ly (gamma(t+1) - gamma(t)),
// and the same for t+1.  The streaming shift of Delta_t is split into an
// integer part di and fraction w, with the nearest-source choices for the two
// boundary planes precomputed so that every kernel makes the same decision.
struct Proto {
  long long t;
  double delta, delta_c, ule;
  double delta_n, delta_nc, ule_n;
  int di, near_lo, near_hi, pad;
  double w;
  float wf_lo, wf_hi;          // interpolation weight on c1 for y = 0 / y = ny-1 receivers
  float delta_f, ule_f;        // FP32 copies of delta and ule
  int kind, ny;
  double rate, gamma0, omega, theta;
};

__device__ inline double proto_increment(const Proto& s, long long t) {
  if (s.kind == 0) return (double)s.ny * s.rate;
  double a = s.omega * (double)t + s.theta;
  double b = s.omega * (double)(t + 1) + s.theta;
  return (double)s.ny * s.gamma0 * (cos(a) - cos(b));
}

// Per-box step sums are accumulated with FP64 atomics in L2.  Hundreds of
// blocks or warps adding to the same 34 addresses serialise on them, so each
// adder takes one of ACC_REP replicas (on separate cache lines), chosen by its
// block or particle index; the finalisation adds the replicas.
constexpr int ACC_REP = 16;
constexpr int ACC_STRIDE = 48;   // doubles per replica (40 used)

// Pair-force constants of a box in one compute type (built on the host in
// both types, so that no kernel converts them per pair).
template <typename T>
struct PairConst {
  T kn, kt, eta_n, mu, F0, debye, debye10, lub_cut, lub_delta, eta0, hrange;
  bool rep, lub;   // double-layer force on (F0 > 0), lubrication on (cut-off > 0)
};

// ------------------------------------------------------------ state view
struct View {
  // lattice
  int nx, ny, nz;
  long long ncell;
  double tau, rho0, g[3];
  int has_g;                    // nonzero body force
  float inv_scale, scale;       // deviation storage scale (P = 2, 3)
  // per-node constants in both precisions (no FP64 arithmetic on the FP32 paths)
  double omega_d, vf_d;         // 1/tau and -(1 - 1/(2 tau))
  float omega_f, vf_f, rho0_f, g_f[3];
  int ladd;                     // Ladd's operator instead of BGK
  double ls_d, lb_d, vfb_d;     // Ladd: 1 + lambda, 1 + lambda_v (lambda = -1/tau, lambda_v = -1/tau_bulk),
  float ls_f, lb_f, vfb_f;      //  and -(1 + lambda_v / 2) for the bulk viscous stress
  double inv_nx_d, inv_ny_d, inv_nz_d;   // reciprocal box lengths
  float inv_nx_f, inv_ny_f, inv_nz_f;
  void* fa;                     // population buffers; step t reads fa when t is even
  void* fb;
  double* step_acc;             // [ACC_REP][ACC_STRIDE] replicas of the 40 sums of the current step:
                                //  0-5 viscous (xx yy zz xy xz yz), 6-14 stresslet, 15-23 contact
                                //  virial, 24 contacts, 25-33 repulsive, 34-39 lubrication stresslets
  int* owner;                   // -1 fluid, else particle
  void* plane_mom;              // [2][nz][nx] (rho, jx, jy, jz) in compute type, of the populations
  void* plane_mom2;             //  read at even (plane_mom) and odd (plane_mom2) step counts
  // particles
  int n;
  double *R, *U, *W, *rad, *amap, *mass, *inert, *inv_m, *inv_I;
  double *R2, *U2, *W2;           // second state buffer of the particle sub-steps
  // FP32 compute: per particle the step-start centre Ro (FP64) and, for each
  // state buffer, an FP32 mirror [n][12] of (R - Ro, U, W) (pads at 3, 7, 11)
  // that the partners read; per candidate (canonical pair a < b) the
  // step-start displacement D = R_b - R_a (minimum image, FP32) with
  // c0 = |D|^2 - (a_a + a_b)^2 (taken in FP64), and the image index k
  double* Ro;
  float* m32[2];
  float4* pd;                     // [n][PAIR_SLOTS] (D, c0)
  signed char* pk;                // [n][PAIR_SLOTS]
  int* pcx;                       // [n][8] cell of each particle at the step start (x, y, z, x of the rows across the planes)
  void* plb;                    // [n][12] compute-type copy: R, U, W, radius (and pad)
  double *Fh, *Th, *Fcov, *Tcov, *Fp, *Tp;
  // cell list
  int ncx, ncy, ncz, brute;
  double csx, csy, csz, inv_csx, inv_csy, inv_csz;
  int *cell_start, *cell_cnt, *cell_ids, *pcell;
  int ncells;
  // per-step candidate partners and their springs: [n][PAIR_SLOTS]
  int* pj;
  double* ph;                   // [n][PAIR_SLOTS][3]
  int* pcnt;                    // [n]
  int* drv;                     // [n] 1: driven sphere (keeps its velocity and spin)
  int has_drv;                  // some sphere is driven
  void* pconst;                 // [n][8] per-step constants in the compute type: F^h + F^cov,
                                //  T^h + T^cov, 1 / m, 1 / I (written at the step start)
  // tangential-spring table: per particle a, partners b > a
  int K;
  int *hcnt0, *hpart0, *hcnt1, *hpart1;
  double *hval0, *hval1;
  // physics
  double mu, kn, kt, eta_n, F0, debye, lub_delta, lub_cut, eta0, hrange;
  int nsub, quasi2d, move, nbins;
  double dt_sub;                // 1 / nsub
  PairConst<double> pc_d;       // the pair constants above in each compute type
  PairConst<float> pc_f;
  // accumulators
  double* sums;                 // [4][9] Kahan sums (visc, slet, contact, repulsive) + [4][9] comps
  double* hist;                 // [3 nbins]
  unsigned long long* counters; // [0] samples, [1] contacts
  Proto* proto;
  int* err;
  // three tensor maps (CUtensorMap, 128 bytes each) for the staged
  // collide-stream: the population buffers fa, fb as [19][nz][ny][nx] and the
  // owner words; NULL when the box has none (FP64 storage, or x rows not a
  // multiple of 16 bytes)
  const void* tmap;
  // [n][12] the compute-type copy of the next step, written by the particle
  // kernel while the collide-stream still reads plb beside it (the
  // finalisation then copies it into plb)
  void* plb_next;
};

// ERR_LINKS: a particle has more surface nodes than the link kernel stages.
// Candidate partners per particle and lattice step (two per lane of a warp).
constexpr int PAIR_SLOTS = 64;
// Tangential springs per particle in the step tables (partners with larger index).
constexpr int HSLOTS_DEV = 16;
// Boxes with at most this many particles find candidates by scanning all
// particles instead of through the cell list.
constexpr int BRUTE_PAIRS_MAX = 4096;

// ERR_TIMEOUT: a bounded device wait gave up (the step's results are invalid).
enum ErrBits { ERR_OVERLAP = 1, ERR_UNSTABLE = 2, ERR_LINKS = 4, ERR_PAIRS = 8, ERR_TIMEOUT = 16 };

// Replica r (taken modulo ACC_REP) of a box's step sums.
__device__ __forceinline__ double* acc_rep(const View& v, int r) {
  return v.step_acc + (r & (ACC_REP - 1)) * ACC_STRIDE;
}

// A set of boxes stepped together (one box for the single-box API).  Work of
// every kernel is numbered across the boxes; the prefix tables map a global
// work index (collide-stream tile, particle, plane node, cell) to its box.
struct Batch {
  const View* __restrict__ views;   // [nbox], device
  const int* __restrict__ tile_off;   // [nbox + 1] collide-stream tiles (32 x 2^tile_lg nodes)
  const int* __restrict__ part_off;   // [nbox + 1] particles
  const int* __restrict__ plane_off;  // [nbox + 1] Lees-Edwards plane nodes (2 nx nz)
  const int* __restrict__ cell_off;   // [nbox + 1] cell-list cells
  int nbox;
  int max_nsub;
  int tile_lg;                        // collide-stream tile height: 2^tile_lg rows
  int dem_fin;                        // the particle kernel ends with the step's finalisation
};

// Box owning global work index g (off is an ascending prefix table).
__device__ __forceinline__ int box_of(const int* __restrict__ off, int nbox, int g) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Select the double or float copy of a constant for compute type T.
template <typename T> __device__ __forceinline__ T sel(double d, float f);
template <> __device__ __forceinline__ double sel<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float sel<float>(double, float f) { return f; }

// Population buffer holding n*(t) for the box's current step counter.
__device__ __forceinline__ void* fin_of(const View& v) { return (v.proto->t & 1) ? v.fb : v.fa; }
__device__ __forceinline__ void* fout_of(const View& v) { return (v.proto->t & 1) ? v.fa : v.fb; }
// Lees-Edwards plane moments of fin_of(v) (read by the crossing pulls) and of
// fout_of(v) (written by the collide-stream for the next step).
__device__ __forceinline__ void* pm_in_of(const View& v) { return (v.proto->t & 1) ? v.plane_mom2 : v.plane_mom; }
__device__ __forceinline__ void* pm_out_of(const View& v) { return (v.proto->t & 1) ? v.plane_mom : v.plane_mom2; }

__host__ __device__ inline int wrapi(int v, int L) { int r = v % L; return r < 0 ? r + L : r; }
// Periodic wrap of an index at most one period outside [0, L).
__host__ __device__ __forceinline__ int wrap1(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Lees-Edwards minimum image of d = p - R for a particle centre R: returns k,
// the image R + k (delta, ny, 0) moving with U + k U_LE e_x.  Multiplies by the
// reciprocal box lengths (no division on the hot paths).
template <typename T>
__device__ inline int le_image(T& dx, T& dy, T& dz, T delta, int nx, int ny, int nz, T ix, T iy,
                               T iz) {
  const T fny = (T)ny, fnx = (T)nx, fnz = (T)nz;
  int k = (int)floor(dy * iy + (T)0.5);
  dy -= (T)k * fny;
  dx -= (T)k * delta;
  dx -= fnx * floor(dx * ix + (T)0.5);
  dz -= fnz * floor(dz * iz + (T)0.5);
  return k;
}

template <typename T>
__device__ inline int le_image_v(const View& v, T& dx, T& dy, T& dz, T delta) {
  return le_image<T>(dx, dy, dz, delta, v.nx, v.ny, v.nz, sel<T>(v.inv_nx_d, v.inv_nx_f),
                     sel<T>(v.inv_ny_d, v.inv_ny_f), sel<T>(v.inv_nz_d, v.inv_nz_f));
}

// Lattice weight C^q for a runtime direction.
__host__ __device__ inline float wq_f(int q) { return q == 0 ? 1.0f / 3.0f : (q <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f); }
__host__ __device__ inline double wq_d(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
template <typename T> __device__ inline T wq(int q);
template <> __device__ inline float wq<float>(int q) { return wq_f(q); }
template <> __device__ inline double wq<double>(int q) { return wq_d(q); }

template <typename T>
__device__ inline T feq(int q, T rho, T jx, T jy, T jz, T inv_rho) {
  T jc = jx * (T)D3Q19::cx(q) + jy * (T)D3Q19::cy(q) + jz * (T)D3Q19::cz(q);
  T jj = jx * jx + jy * jy + jz * jz;
  return (T)D3Q19::w(q) * (rho + (T)3 * jc + (T)4.5 * jc * jc * inv_rho - (T)1.5 * jj * inv_rho);
}

// Sum over the 32 lanes of a warp (fixed order).
__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide sum of NV values held by every thread (blockDim multiple of 32,
// <= 1024); result valid in thread 0.  Fixed reduction order.
template <typename T, int NV>
__device__ inline void block_sum(T (&v)[NV], T* smem /* [32][NV] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[wid * NV + k] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = lane < nw ? smem[lane * NV + k] : (T)0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
  }
  __syncthreads();
}

}  // namespace susp_dev
