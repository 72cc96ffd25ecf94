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
  x -= v.nx * floor(x / v.nx);
  z -= v.nz * floor(z / v.nz);
  int cx = (int)floor(x / v.csx), cy = (int)floor(y / v.csy), cz = (int)floor(z / v.csz);
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

__device__ inline void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ inline double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

struct PairOut {
  double Fa[3], Ta[3], Tb[3];   // total pair force on a (b gets -Fa), torques
  double Fc[3];                 // contact part of Fa (for the virial)
  double Fr[3];                 // double-layer part of Fa
  double ht[3];                 // updated tangential spring
  double fn;                    // normal-force magnitude (repulsive positive)
  double d[3];                  // R_b - R_a (minimum image)
  int touching;
};

// Full interaction of the canonical pair (a, b); returns false if out of range.
__device__ bool pair_interact(const View& v, int a, int b, const int* hcnt, const int* hpart,
                              const double* hval, double delta, double ule, double dt, PairOut& o) {
  double d[3] = {v.R[3 * b] - v.R[3 * a], v.R[3 * b + 1] - v.R[3 * a + 1], v.R[3 * b + 2] - v.R[3 * a + 2]};
  const int k = (int)floor(d[1] / v.ny + 0.5);
  d[1] -= k * (double)v.ny;
  d[0] -= k * delta;
  d[0] -= v.nx * floor(d[0] / v.nx + 0.5);
  d[2] -= v.nz * floor(d[2] / v.nz + 0.5);
  const double ra = v.rad[a], rb = v.rad[b];
  const double dist = sqrt(dot3(d, d));
  const double h = dist - ra - rb;
  if (!(h < v.hrange) && !(h < 0.0)) return false;
  const double uab[3] = {v.U[3 * a] - v.U[3 * b] - k * ule, v.U[3 * a + 1] - v.U[3 * b + 1],
                         v.U[3 * a + 2] - v.U[3 * b + 2]};
  const double* wa = v.W + 3 * a;
  const double* wb = v.W + 3 * b;
  const double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
  for (int c = 0; c < 3; ++c) {
    o.Fa[c] = o.Ta[c] = o.Tb[c] = o.Fc[c] = o.Fr[c] = o.ht[c] = 0.0;
    o.d[c] = d[c];
  }
  o.fn = 0.0;
  o.touching = 0;
  // ---- contact
  const double overlap = ra + rb - dist;
  if (overlap > 0.0) {
    double ht[3] = {0.0, 0.0, 0.0};
    const int m = hcnt[a];
    for (int s = 0; s < m; ++s)
      if (hpart[a * v.K + s] == b) {
        for (int c = 0; c < 3; ++c) ht[c] = hval[3 * (a * v.K + s) + c];
        break;
      }
    const double ws[3] = {ra * wa[0] + rb * wb[0], ra * wa[1] + rb * wb[1], ra * wa[2] + rb * wb[2]};
    double rot[3];
    cross3(ws, n, rot);
    const double vv[3] = {uab[0] + rot[0], uab[1] + rot[1], uab[2] + rot[2]};
    const double vn = dot3(vv, n);
    const double vt[3] = {vv[0] - vn * n[0], vv[1] - vn * n[1], vv[2] - vn * n[2]};
    const double fn = v.kn * overlap + v.eta_n * vn;
    const double hn = dot3(ht, n);
    for (int c = 0; c < 3; ++c) ht[c] = ht[c] - hn * n[c] + vt[c] * dt;
    double ft[3] = {-v.kt * ht[0], -v.kt * ht[1], -v.kt * ht[2]};
    const double ftm = sqrt(dot3(ft, ft));
    const double cap = v.mu * fabs(fn);
    if (ftm >= cap && ftm > 0.0) {
      for (int c = 0; c < 3; ++c) {
        ft[c] = cap * ft[c] / ftm;
        ht[c] = -ft[c] / v.kt;
      }
    }
    double tq[3];
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
  if (v.F0 > 0.0 && h < 10.0 * v.debye) {
    const double fr = v.F0 * exp(-(h > 0.0 ? h : 0.0) / v.debye);
    for (int c = 0; c < 3; ++c) {
      o.Fr[c] = -fr * n[c];
      o.Fa[c] += o.Fr[c];
    }
  }
  // ---- lubrication correction
  if (v.lub_cut > 0.0 && h < v.lub_cut) {
    const double hh = h < 0.0 ? 0.0 : h;
    const double sc = 2.0 / (ra + rb);
    const double xi = sc * hh, xc = sc * v.lub_cut, dl = sc * v.lub_delta;
    const double inv = 1.0 / (xi + dl) - 1.0 / (xc + dl);
    const double lg = log((xc + dl) / (xi + dl));
    const double be = rb / ra, bj = ra / rb;
    const double pi = 3.14159265358979323846;
    const double e0 = v.eta0;
    const double op = 1.0 + be, oq = 1.0 + bj;
    const double XA = e0 * 6.0 * pi * ra * (2.0 * be * be / (op * op * op)) * inv;
    const double YA = e0 * 6.0 * pi * ra * (4.0 * be * (2.0 + be + 2.0 * be * be) / (15.0 * op * op * op)) * lg;
    const double YBa = e0 * 4.0 * pi * ra * ra * (be * (4.0 + be) / (5.0 * op * op)) * lg;
    const double YBb = e0 * 4.0 * pi * rb * rb * (bj * (4.0 + bj) / (5.0 * oq * oq)) * lg;
    const double YCaa = e0 * 8.0 * pi * ra * ra * ra * (2.0 * be / (5.0 * op)) * lg;
    const double YCbb = e0 * 8.0 * pi * rb * rb * rb * (2.0 * bj / (5.0 * oq)) * lg;
    const double YCab = e0 * 8.0 * pi * ra * ra * ra * (be * be / (10.0 * op)) * lg;
    const double un = dot3(uab, n);
    double wan[3], wbn[3], nxu[3];
    cross3(wa, n, wan);
    cross3(wb, n, wbn);
    cross3(n, uab, nxu);
    const double wap = dot3(wa, n), wbp = dot3(wb, n);
    for (int c = 0; c < 3; ++c) {
      const double ut = uab[c] - un * n[c];
      o.Fa[c] += -XA * un * n[c] - YA * ut - YBa * wan[c] - YBb * wbn[c];
      const double wat = wa[c] - wap * n[c], wbt = wb[c] - wbp * n[c];
      o.Ta[c] += -YBa * nxu[c] - YCaa * wat - YCab * wbt;
      o.Tb[c] += -YBb * nxu[c] - YCbb * wbt - YCab * wat;
    }
  }
  return true;
}

__global__ void __launch_bounds__(128) k_pairs(View v, const int* __restrict__ hcnt_old,
                                               const int* __restrict__ hpart_old,
                                               const double* __restrict__ hval_old, int* hcnt_new,
                                               int* hpart_new, double* hval_new, double dt, int sample) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const Proto* pr = v.proto;
  const double delta = pr->delta, ule = pr->ule;
  double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
  double cv[9], rv[9];
  for (int c = 0; c < 9; ++c) { cv[c] = 0.0; rv[c] = 0.0; }
  int nnew = 0, ncont = 0;
  const double pi = 3.14159265358979323846;
  const double dth = pi / v.nbins;

  auto visit = [&](int j) {
    if (j == i) return;
    const int a = i < j ? i : j, b = i < j ? j : i;
    PairOut o;
    if (!pair_interact(v, a, b, hcnt_old, hpart_old, hval_old, delta, ule, dt, o)) return;
    if (i == a) {
      for (int c = 0; c < 3; ++c) { F[c] += o.Fa[c]; T[c] += o.Ta[c]; }
      if (o.touching) {
        if (nnew < v.K) {
          hpart_new[a * v.K + nnew] = b;
          for (int c = 0; c < 3; ++c) hval_new[3 * (a * v.K + nnew) + c] = o.ht[c];
          ++nnew;
        } else {
          atomicOr(v.err, ERR_PAIRS);
        }
      }
      if (sample) {
        const double r[3] = {-o.d[0], -o.d[1], -o.d[2]};
        if (o.touching) {
          for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) cv[3 * x + y] += 0.5 * (r[x] * o.Fc[y] + r[y] * o.Fc[x]);
          double th = atan2(r[1], r[0]);
          const double tx = -sin(th), ty = cos(th);
          if (th < 0.0) th += pi;
          if (th >= pi) th -= pi;
          int bin = (int)floor(th / dth);
          if (bin >= v.nbins) bin = v.nbins - 1;
          if (bin < 0) bin = 0;
          atomicAdd(v.hist + 3 * bin, 1.0);
          atomicAdd(v.hist + 3 * bin + 1, o.fn);
          atomicAdd(v.hist + 3 * bin + 2, o.Fc[0] * tx + o.Fc[1] * ty);
          ++ncont;
        }
        if (v.F0 > 0.0)
          for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) rv[3 * x + y] += 0.5 * (r[x] * o.Fr[y] + r[y] * o.Fr[x]);
      }
    } else {
      for (int c = 0; c < 3; ++c) { F[c] -= o.Fa[c]; T[c] += o.Tb[c]; }
    }
  };

  if (v.brute) {
    for (int j = 0; j < v.n; ++j) visit(j);
  } else {
    double x = v.R[3 * i], y = v.R[3 * i + 1], z = v.R[3 * i + 2];
    x -= v.nx * floor(x / v.nx);
    z -= v.nz * floor(z / v.nz);
    const int cy = min(max((int)floor(y / v.csy), 0), v.ncy - 1);
    const int cz = min(max((int)floor(z / v.csz), 0), v.ncz - 1);
    const int zlo = v.ncz >= 3 ? -1 : 0, zhi = v.ncz >= 2 ? 1 : 0;
    for (int dy = -1; dy <= 1; ++dy) {
      int yc = cy + dy;
      double xs = x;
      if (yc < 0) { yc += v.ncy; xs = x + delta; }
      else if (yc >= v.ncy) { yc -= v.ncy; xs = x - delta; }
      xs -= v.nx * floor(xs / v.nx);
      const int cxs = min(max((int)floor(xs / v.csx), 0), v.ncx - 1);
      for (int dx = -1; dx <= 1; ++dx) {
        const int xc = wrapi(cxs + dx, v.ncx);
        for (int dz = zlo; dz <= zhi; ++dz) {
          const int zc = wrapi(cz + dz, v.ncz);
          const int c = xc + v.ncx * (yc + v.ncy * zc);
          const int s = v.cell_start[c], e = v.cell_start[c + 1];
          for (int t = s; t < e; ++t) visit(v.cell_ids[t]);
        }
      }
    }
  }
  for (int c = 0; c < 3; ++c) { v.Fp[3 * i + c] = F[c]; v.Tp[3 * i + c] = T[c]; }
  hcnt_new[i] = nnew;
  if (sample) {
    for (int c = 0; c < 9; ++c) { v.cvir_part[9 * i + c] = cv[c]; v.rvir_part[9 * i + c] = rv[c]; }
    v.ncont_part[i] = ncont;
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
  const double m = v.mass[i], I = v.inert[i];
  for (int c = 0; c < 3; ++c) {
    const double F = v.Fh[3 * i + c] + v.Fcov[3 * i + c] + v.Fp[3 * i + c];
    const double T = v.Th[3 * i + c] + v.Tcov[3 * i + c] + v.Tp[3 * i + c];
    U[c] += dt * F / m;
    W[c] += dt * T / I;
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

// One particle sub-step: cell list, pair interactions, integration.
void launch_dem_substep(const View& v, int parity, int sub, int plb_double, cudaStream_t s) {
  if (v.n == 0) return;
  const int nb = (v.n + 127) / 128;
  if (!v.brute) {
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
  k_pairs<<<nb, 128, 0, s>>>(v, hc_old, hp_old, hv_old, hc_new, hp_new, hv_new, dt, sub == 0);
  k_integrate<<<nb, 128, 0, s>>>(v, dt, sub == v.nsub - 1, plb_double);
}
