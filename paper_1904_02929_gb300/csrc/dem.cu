// dem.cu — particle sub-steps: cell list, pair interactions, integration.
//
// Pair interactions (one thread per particle, gathering over the 27 cells
// around it; every pair is evaluated by both partners in the canonical
// orientation a = min(i, j), b = max(i, j) so the two results are bitwise
// equal and opposite, with no atomics):
//   contact (Sec. 2, Eq. 11, 11t): F_n = kn delta_n + eta_n v_n along -n,
//     tangential spring delta_t (kept per pair in a table owned by a),
//     rotated into the tangent plane and advanced by v_t dt, F_t = -kt delta_t
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
#include "susp_dev.cuh"

namespace susp_dev {

__global__ void k_cell_count(View v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
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
}

// Exclusive scan of the cell counts (one block of 1024 threads).
__global__ void k_cell_scan(View v) {
  __shared__ int part[1024];
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

__global__ void k_cell_fill(View v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int c = v.pcell[i];
  const int slot = atomicAdd(v.cell_cnt + c, 1);
  v.cell_ids[v.cell_start[c] + slot] = i;
}

// Sort each cell's ids ascending so the gather order is deterministic.
__global__ void k_cell_sort(View v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.ncells) return;
  const int s = v.cell_start[c], e = v.cell_start[c + 1];
  for (int a = s + 1; a < e; ++a) {
    const int key = v.cell_ids[a];
    int b = a - 1;
    while (b >= s && v.cell_ids[b] > key) { v.cell_ids[b + 1] = v.cell_ids[b]; --b; }
    v.cell_ids[b + 1] = key;
  }
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
  T d[3];                  // R_b - R_a (minimum image)
  int touching;
};

// Minimum-image displacement R_b - R_a in FP64 (positions are FP64 on every
// path); returns false when the pair is out of range.
__device__ inline bool pair_geometry(const View& v, int a, int b, double delta, double d[3], int& k,
                                     double& h) {
  d[0] = v.R[3 * b] - v.R[3 * a];
  d[1] = v.R[3 * b + 1] - v.R[3 * a + 1];
  d[2] = v.R[3 * b + 2] - v.R[3 * a + 2];
  k = (int)floor(d[1] * v.inv_ny_d + 0.5);
  d[1] -= k * (double)v.ny;
  d[0] -= k * delta;
  d[0] -= v.nx * floor(d[0] * v.inv_nx_d + 0.5);
  d[2] -= v.nz * floor(d[2] * v.inv_nz_d + 0.5);
  const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double rsum = v.rad[a] + v.rad[b];
  const double lim = rsum + v.hrange + 1e-9;
  if (!(d2 < lim * lim)) return false;   // cheap rejection before the square root
  h = sqrt(d2) - rsum;
  return (h < v.hrange) || (h < 0.0);
}

// Full interaction of the canonical pair (a, b) in precision T, given the
// minimum-image displacement.
template <typename T>
__device__ void pair_interact(const View& v, int a, int b, const double dd[3], int k, double hd,
                              const int* hcnt, const int* hpart, const double* hval, T ule, T dt,
                              PairOut<T>& o) {
  const T d[3] = {(T)dd[0], (T)dd[1], (T)dd[2]};
  const T ra = (T)v.rad[a], rb = (T)v.rad[b];
  const T dist = sqrt(dot3(d, d));
  const T h = (T)hd;
  const T uab[3] = {(T)(v.U[3 * a] - v.U[3 * b]) - (T)k * ule, (T)(v.U[3 * a + 1] - v.U[3 * b + 1]),
                    (T)(v.U[3 * a + 2] - v.U[3 * b + 2])};
  const T wa[3] = {(T)v.W[3 * a], (T)v.W[3 * a + 1], (T)v.W[3 * a + 2]};
  const T wb[3] = {(T)v.W[3 * b], (T)v.W[3 * b + 1], (T)v.W[3 * b + 2]};
  const T n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
  for (int c = 0; c < 3; ++c) {
    o.Fa[c] = o.Ta[c] = o.Tb[c] = o.Fc[c] = o.Fr[c] = o.ht[c] = (T)0;
    o.d[c] = d[c];
  }
  o.fn = (T)0;
  o.touching = 0;
  // ---- contact
  const T overlap = ra + rb - dist;
  if (hd < 0.0) {
    T ht[3] = {0, 0, 0};
    const int m = hcnt[a];
    for (int s = 0; s < m; ++s)
      if (hpart[a * v.K + s] == b) {
        for (int c = 0; c < 3; ++c) ht[c] = (T)hval[3 * (a * v.K + s) + c];
        break;
      }
    const T ws[3] = {ra * wa[0] + rb * wb[0], ra * wa[1] + rb * wb[1], ra * wa[2] + rb * wb[2]};
    T rot[3];
    cross3(ws, n, rot);
    const T vv[3] = {uab[0] + rot[0], uab[1] + rot[1], uab[2] + rot[2]};
    const T vn = dot3(vv, n);
    const T vt[3] = {vv[0] - vn * n[0], vv[1] - vn * n[1], vv[2] - vn * n[2]};
    const T kn = (T)v.kn, kt = (T)v.kt;
    const T fn = kn * overlap + (T)v.eta_n * vn;
    const T hn = dot3(ht, n);
    for (int c = 0; c < 3; ++c) ht[c] = ht[c] - hn * n[c] + vt[c] * dt;
    T ft[3] = {-kt * ht[0], -kt * ht[1], -kt * ht[2]};
    const T ftm = sqrt(dot3(ft, ft));
    const T cap = (T)v.mu * fabs(fn);
    if (ftm >= cap && ftm > (T)0) {
      for (int c = 0; c < 3; ++c) {
        ft[c] = cap * ft[c] / ftm;
        ht[c] = -ft[c] / kt;
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
  if (v.F0 > 0.0 && hd < 10.0 * v.debye) {
    const T fr = (T)v.F0 * exp(-(h > (T)0 ? h : (T)0) / (T)v.debye);
    for (int c = 0; c < 3; ++c) {
      o.Fr[c] = -fr * n[c];
      o.Fa[c] += o.Fr[c];
    }
  }
  // ---- lubrication correction
  if (v.lub_cut > 0.0 && hd < v.lub_cut) {
    const T hh = h < (T)0 ? (T)0 : h;
    const T sc = (T)2 / (ra + rb);
    const T xi = sc * hh, xc = sc * (T)v.lub_cut, dl = sc * (T)v.lub_delta;
    const T inv = (T)1 / (xi + dl) - (T)1 / (xc + dl);
    const T lg = log((xc + dl) / (xi + dl));
    const T be = rb / ra, bj = ra / rb;
    const T pi = (T)3.14159265358979323846;
    const T e0 = (T)v.eta0;
    const T op = (T)1 + be, oq = (T)1 + bj;
    const T XA = e0 * (T)6 * pi * ra * ((T)2 * be * be / (op * op * op)) * inv;
    const T YA = e0 * (T)6 * pi * ra * ((T)4 * be * ((T)2 + be + (T)2 * be * be) / ((T)15 * op * op * op)) * lg;
    const T YBa = e0 * (T)4 * pi * ra * ra * (be * ((T)4 + be) / ((T)5 * op * op)) * lg;
    const T YBb = e0 * (T)4 * pi * rb * rb * (bj * ((T)4 + bj) / ((T)5 * oq * oq)) * lg;
    const T YCaa = e0 * (T)8 * pi * ra * ra * ra * ((T)2 * be / ((T)5 * op)) * lg;
    const T YCbb = e0 * (T)8 * pi * rb * rb * rb * ((T)2 * bj / ((T)5 * oq)) * lg;
    const T YCab = e0 * (T)8 * pi * ra * ra * ra * (be * be / ((T)10 * op)) * lg;
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
  }
}

template <typename T>
__device__ inline T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// One warp per particle i; the lanes split the candidate partners (one
// neighbour cell per lane, or a strided slice of all particles in brute-force
// mode).  Forces are summed per lane and reduced across the warp.
template <typename T>
__global__ void __launch_bounds__(128) k_pairs(View v, const int* __restrict__ hcnt_old,
                                               const int* __restrict__ hpart_old,
                                               const double* __restrict__ hval_old, int* hcnt_new,
                                               int* hpart_new, double* hval_new, double dt_d, int sample) {
  __shared__ int s_slot[4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * 4 + wib;
  if (lane == 0) s_slot[wib] = 0;
  __syncwarp();
  if (i >= v.n) return;
  const Proto* pr = v.proto;
  const double delta = pr->delta;
  const T ule = (T)pr->ule;
  const T dt = (T)dt_d;
  T F[3] = {0, 0, 0}, Tq[3] = {0, 0, 0};
  T cv[9], rv[9];
  for (int c = 0; c < 9; ++c) { cv[c] = (T)0; rv[c] = (T)0; }
  int ncont = 0;
  const double pi = 3.14159265358979323846;
  const double dth = pi / v.nbins;

  auto visit = [&](int j) {
    if (j == i) return;
    const int a = i < j ? i : j, b = i < j ? j : i;
    double dd[3], hd;
    int k;
    if (!pair_geometry(v, a, b, delta, dd, k, hd)) return;
    PairOut<T> o;
    pair_interact<T>(v, a, b, dd, k, hd, hcnt_old, hpart_old, hval_old, ule, dt, o);
    if (i == a) {
      for (int c = 0; c < 3; ++c) { F[c] += o.Fa[c]; Tq[c] += o.Ta[c]; }
      if (o.touching) {
        const int slot = atomicAdd(&s_slot[wib], 1);
        if (slot < v.K) {
          hpart_new[a * v.K + slot] = b;
          for (int c = 0; c < 3; ++c) hval_new[3 * (a * v.K + slot) + c] = (double)o.ht[c];
        } else {
          atomicOr(v.err, ERR_PAIRS);
        }
      }
      if (sample) {
        const T r[3] = {-o.d[0], -o.d[1], -o.d[2]};
        if (o.touching) {
          for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) cv[3 * x + y] += (T)0.5 * (r[x] * o.Fc[y] + r[y] * o.Fc[x]);
          double th = atan2((double)r[1], (double)r[0]);
          const double tx = -sin(th), ty = cos(th);
          if (th < 0.0) th += pi;
          if (th >= pi) th -= pi;
          int bin = (int)floor(th / dth);
          if (bin >= v.nbins) bin = v.nbins - 1;
          if (bin < 0) bin = 0;
          atomicAdd(v.hist + 3 * bin, 1.0);
          atomicAdd(v.hist + 3 * bin + 1, (double)o.fn);
          atomicAdd(v.hist + 3 * bin + 2, (double)o.Fc[0] * tx + (double)o.Fc[1] * ty);
          ++ncont;
        }
        if (v.F0 > 0.0)
          for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) rv[3 * x + y] += (T)0.5 * (r[x] * o.Fr[y] + r[y] * o.Fr[x]);
      }
    } else {
      for (int c = 0; c < 3; ++c) { F[c] -= o.Fa[c]; Tq[c] += o.Tb[c]; }
    }
  };

  if (v.brute) {
    for (int j = lane; j < v.n; j += 32) visit(j);
  } else if (lane < 27) {
    const int dyc = lane / 9 - 1, dxc = (lane / 3) % 3 - 1, dzc = lane % 3 - 1;
    const int zlo = v.ncz >= 3 ? -1 : 0, zhi = v.ncz >= 2 ? 1 : 0;
    if (dzc >= zlo && dzc <= zhi) {
      double x = v.R[3 * i], y = v.R[3 * i + 1], z = v.R[3 * i + 2];
      x -= v.nx * floor(x * v.inv_nx_d);
      z -= v.nz * floor(z * v.inv_nz_d);
      const int cy = min(max((int)floor(y * v.inv_csy), 0), v.ncy - 1);
      const int cz = min(max((int)floor(z * v.inv_csz), 0), v.ncz - 1);
      int yc = cy + dyc;
      double xs = x;
      if (yc < 0) { yc += v.ncy; xs = x + delta; }
      else if (yc >= v.ncy) { yc -= v.ncy; xs = x - delta; }
      xs -= v.nx * floor(xs * v.inv_nx_d);
      const int cxs = min(max((int)floor(xs * v.inv_csx), 0), v.ncx - 1);
      const int xc = wrapi(cxs + dxc, v.ncx);
      const int zc = wrapi(cz + dzc, v.ncz);
      const int c = xc + v.ncx * (yc + v.ncy * zc);
      const int s0 = v.cell_start[c], e0 = v.cell_start[c + 1];
      for (int t = s0; t < e0; ++t) visit(v.cell_ids[t]);
    }
  }
  for (int c = 0; c < 3; ++c) { F[c] = warp_sum(F[c]); Tq[c] = warp_sum(Tq[c]); }
  if (sample) {
    for (int c = 0; c < 9; ++c) { cv[c] = warp_sum(cv[c]); rv[c] = warp_sum(rv[c]); }
    for (int o = 16; o > 0; o >>= 1) ncont += __shfl_xor_sync(0xffffffffu, ncont, o);
  }
  __syncwarp();
  if (lane == 0) {
    for (int c = 0; c < 3; ++c) { v.Fp[3 * i + c] = (double)F[c]; v.Tp[3 * i + c] = (double)Tq[c]; }
    const int m = s_slot[wib];
    hcnt_new[i] = m < v.K ? m : v.K;
    if (sample) {
      for (int c = 0; c < 9; ++c) { v.cvir_part[9 * i + c] = (double)cv[c]; v.rvir_part[9 * i + c] = (double)rv[c]; }
      v.ncont_part[i] = ncont;
    }
  }
}

template <typename TC>
__device__ inline void write_plb(const View& v, int i) {
  TC* pp = reinterpret_cast<TC*>(v.plb) + 12 * i;
  for (int c = 0; c < 3; ++c) {
    pp[c] = (TC)v.R[3 * i + c];
    pp[3 + c] = (TC)v.U[3 * i + c];
    pp[6 + c] = (TC)v.W[3 * i + c];
  }
}

__global__ void k_integrate(View v, double dt, int last, int plb_double) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  double* R = v.R + 3 * i;
  double* U = v.U + 3 * i;
  double* W = v.W + 3 * i;
  const double im = v.inv_m[i], iI = v.inv_I[i];
  for (int c = 0; c < 3; ++c) {
    const double F = v.Fh[3 * i + c] + v.Fcov[3 * i + c] + v.Fp[3 * i + c];
    const double T = v.Th[3 * i + c] + v.Tcov[3 * i + c] + v.Tp[3 * i + c];
    U[c] += dt * F * im;
    W[c] += dt * T * iI;
  }
  if (v.quasi2d) { U[2] = 0.0; W[0] = 0.0; W[1] = 0.0; }
  for (int c = 0; c < 3; ++c) R[c] += dt * U[c];
  if (!last) return;
  const Proto* pr = v.proto;
  if (R[1] >= v.ny) { R[1] -= v.ny; R[0] -= pr->delta_n; U[0] -= pr->ule; }
  else if (R[1] < 0.0) { R[1] += v.ny; R[0] += pr->delta_n; U[0] += pr->ule; }
  R[0] -= v.nx * floor(R[0] / v.nx);
  R[2] -= v.nz * floor(R[2] / v.nz);
  const double sp = sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
  if (!(sp < 0.5)) atomicOr(v.err, ERR_UNSTABLE);
  if (plb_double) write_plb<double>(v, i);
  else write_plb<float>(v, i);
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

// One particle sub-step: (at sub-step 0) the cell list, then the pair
// interactions and the integration.  The cell list stays valid over the
// sub-steps of a lattice step: the cells are at least one lattice unit larger
// than the interaction range and a particle moves less than 0.5 per step.
void launch_dem_substep(const View& v, int parity, int sub, int plb_double, cudaStream_t s) {
  if (v.n == 0) return;
  const int nb = (v.n + 127) / 128;
  if (!v.brute && sub == 0) {
    cudaMemsetAsync(v.cell_cnt, 0, sizeof(int) * v.ncells, s);
    k_cell_count<<<nb, 128, 0, s>>>(v);
    k_cell_scan<<<1, 1024, 0, s>>>(v);
    k_cell_fill<<<nb, 128, 0, s>>>(v);
    k_cell_sort<<<(v.ncells + 127) / 128, 128, 0, s>>>(v);
  }
  const int* hc_old = parity ? v.hcnt1 : v.hcnt0;
  const int* hp_old = parity ? v.hpart1 : v.hpart0;
  const double* hv_old = parity ? v.hval1 : v.hval0;
  int* hc_new = parity ? v.hcnt0 : v.hcnt1;
  int* hp_new = parity ? v.hpart0 : v.hpart1;
  double* hv_new = parity ? v.hval0 : v.hval1;
  const double dt = 1.0 / v.nsub;
  const int pb = (v.n + 3) / 4;
  if (plb_double)
    k_pairs<double><<<pb, 128, 0, s>>>(v, hc_old, hp_old, hv_old, hc_new, hp_new, hv_new, dt, sub == 0);
  else
    k_pairs<float><<<pb, 128, 0, s>>>(v, hc_old, hp_old, hv_old, hc_new, hp_new, hv_new, dt, sub == 0);
  k_integrate<<<nb, 128, 0, s>>>(v, dt, sub == v.nsub - 1, plb_double);
}
