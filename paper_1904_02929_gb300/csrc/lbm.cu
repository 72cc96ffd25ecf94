// lbm.cu — fused D3Q19 collide-stream kernel (pull scheme, A/B buffers).
//
// Per fluid node r and direction p the post-streaming population is
//   n_p(r, t+1) = n*_p(r - c_p, t)                          (Eq. 3, pull form)
// with three exceptions:
//   * the source r - c_p is solid: moving bounce-back (Eq. 7, 8)
//       n_p(r, t+1) = n*_q(r, t) - 6 C^q rho0 (u_b . c_q),  q = -p,
//       u_b = U + Omega x (r_b - R), r_b = r + c_q / 2;
//   * the source lies beyond a Lees-Edwards plane (y = 0 from below or
//     y = ny-1 from above): the image box is shifted by -/+ Delta in x and
//     moves with -/+ U_LE, so the value is linearly interpolated between the
//     two nodes straddling x - c_px +/- Delta on the opposite plane and
//     Galilean-shifted by n^eq(rho, j -/+ rho U_LE e_x) - n^eq(rho, j);
//     the nearer of the two nodes decides solid (bounce-back) or fluid, and
//     a solid farther node leaves the nearer one alone as the source;
//   * solid nodes are skipped.
// Then the BGK collision (Eq. 4, 5 with every non-conserved mode relaxed by
// 1/tau) and an optional uniform body force 3 C^q (g . c_q).  Each block also
// sums the viscous stress -(1 - 1/(2 tau)) Pi^neq of its fluid nodes.
//
// Bytes per fluid node and step: 19 loads + 19 stores of the storage type
// plus the 4-byte node mask (algorithmic 2 * 19 * s).
#include "susp_dev.cuh"

namespace susp_dev {

template <int P>
__device__ __forceinline__ typename Store<P>::C bounce_value(
    const View& v, const typename Store<P>::C* __restrict__ plb, int i, int x, int y, int z, int q,
    typename Store<P>::C nq_self, typename Store<P>::C delta, typename Store<P>::C ule,
    typename Store<P>::C rho0) {
  using TC = typename Store<P>::C;
  const TC* pp = plb + 12 * i;
  TC dx = (TC)x + (TC)0.5 * (TC)D3Q19::cx(q) - pp[0];
  TC dy = (TC)y + (TC)0.5 * (TC)D3Q19::cy(q) - pp[1];
  TC dz = (TC)z + (TC)0.5 * (TC)D3Q19::cz(q) - pp[2];
  int k = le_image(dx, dy, dz, delta, v.nx, v.ny, v.nz);
  TC ubx = pp[3] + (pp[7] * dz - pp[8] * dy) + (TC)k * ule;
  TC uby = pp[4] + (pp[8] * dx - pp[6] * dz);
  TC ubz = pp[5] + (pp[6] * dy - pp[7] * dx);
  TC cu = ubx * (TC)D3Q19::cx(q) + uby * (TC)D3Q19::cy(q) + ubz * (TC)D3Q19::cz(q);
  return nq_self - (TC)6 * (TC)D3Q19::w(q) * rho0 * cu;
}

// Pull across a Lees-Edwards plane (direction p with c_py = +1 at y = 0, or
// c_py = -1 at y = ny-1).
template <int P, int p>
__device__ __noinline__ typename Store<P>::C le_pull(const View v, const typename Store<P>::T* __restrict__ fin,
                                                     const typename Store<P>::C* __restrict__ plb,
                                                     const Proto* __restrict__ pr, int x, int y, int z,
                                                     long long idx) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  const int nx = v.nx, ny = v.ny;
  const long long nc = v.ncell;
  constexpr int cpx = D3Q19::cx(p), cpy = D3Q19::cy(p), cpz = D3Q19::cz(p);
  constexpr int q = D3Q19::opp(p);
  const bool below = (cpy == 1);
  const int sx = x - cpx, sz = wrapi(z - cpz, v.nz);
  const int ys = below ? ny - 1 : 0;
  const int di = pr->di;
  const int c0x = below ? wrapi(sx + di, nx) : wrapi(sx - di - 1, nx);
  const int c1x = c0x + 1 == nx ? 0 : c0x + 1;
  const int nearsel = below ? pr->near_lo : pr->near_hi;
  TC w1;
  if (P == 0) w1 = (TC)(below ? pr->w : 1.0 - pr->w);
  else w1 = (TC)(below ? pr->wf_lo : pr->wf_hi);
  const long long i0 = c0x + (long long)nx * (ys + (long long)ny * sz);
  const long long i1 = c1x + (long long)nx * (ys + (long long)ny * sz);
  const long long in_ = nearsel ? i1 : i0, io = nearsel ? i0 : i1;
  const TC delta = sel<TC>(pr->delta, pr->delta_f), ule = sel<TC>(pr->ule, pr->ule_f);
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
  const TC base_p = (TC)D3Q19::w(p) * rho0;
  const TC base_q = (TC)D3Q19::w(q) * rho0;
  const int on = v.owner[in_];
  if (on >= 0) {
    TC self = S::load(fin, (long long)q * nc + idx, base_q, (TC)v.inv_scale);
    return bounce_value<P>(v, plb, on, x, y, z, q, self, delta, ule, rho0);
  }
  const TC* pm = reinterpret_cast<const TC*>(v.plane_mom) + (below ? 4LL * v.nz * nx : 0);
  const long long k0 = 4LL * (c0x + (long long)nx * sz), k1 = 4LL * (c1x + (long long)nx * sz);
  TC val, rho, jx, jy, jz;
  if (v.owner[io] >= 0) {
    const long long kn = nearsel ? k1 : k0;
    val = S::load(fin, (long long)p * nc + in_, base_p, (TC)v.inv_scale);
    rho = pm[kn]; jx = pm[kn + 1]; jy = pm[kn + 2]; jz = pm[kn + 3];
  } else {
    const TC a = (TC)1 - w1;
    val = a * S::load(fin, (long long)p * nc + i0, base_p, (TC)v.inv_scale) +
          w1 * S::load(fin, (long long)p * nc + i1, base_p, (TC)v.inv_scale);
    rho = a * pm[k0] + w1 * pm[k1];
    jx = a * pm[k0 + 1] + w1 * pm[k1 + 1];
    jy = a * pm[k0 + 2] + w1 * pm[k1 + 2];
    jz = a * pm[k0 + 3] + w1 * pm[k1 + 3];
  }
  const TC sgn = below ? (TC)-1 : (TC)1;
  const TC inv = (TC)1 / rho;
  val += feq<TC>(p, rho, jx + sgn * rho * ule, jy, jz, inv) - feq<TC>(p, rho, jx, jy, jz, inv);
  return val;
}

template <int P, int p>
__device__ __forceinline__ void pull_one(const View& v, const typename Store<P>::T* __restrict__ fin,
                                         const typename Store<P>::C* __restrict__ plb,
                                         const Proto* __restrict__ pr, uint32_t m, int x, int y,
                                         int z, int xm, int xp, int zm, int zp, long long idx,
                                         typename Store<P>::C delta, typename Store<P>::C ule,
                                         typename Store<P>::C (&n)[19]) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  constexpr int cpx = D3Q19::cx(p), cpy = D3Q19::cy(p), cpz = D3Q19::cz(p);
  constexpr int q = D3Q19::opp(p);
  const int sy = y - cpy;
  if (cpy != 0 && (sy < 0 || sy >= v.ny)) {
    n[p] = le_pull<P, p>(v, fin, plb, pr, x, y, z, idx);
    return;
  }
  const int sx = cpx == 1 ? xm : (cpx == -1 ? xp : x);
  const int sz = cpz == 1 ? zm : (cpz == -1 ? zp : z);
  const long long sidx = sx + (long long)v.nx * (sy + (long long)v.ny * sz);
  const long long nc = v.ncell;
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
  if ((m >> p) & 1u) {
    const int i = v.owner[sidx];
    const TC self = S::load(fin, (long long)q * nc + idx, (TC)D3Q19::w(q) * rho0, (TC)v.inv_scale);
    n[p] = bounce_value<P>(v, plb, i, x, y, z, q, self, delta, ule, rho0);
  } else {
    n[p] = S::load(fin, (long long)p * nc + sidx, (TC)D3Q19::w(p) * rho0, (TC)v.inv_scale);
  }
}

template <int P, int p>
struct PullAll {
  __device__ __forceinline__ static void run(const View& v, const typename Store<P>::T* __restrict__ fin,
                                             const typename Store<P>::C* __restrict__ plb,
                                             const Proto* __restrict__ pr, uint32_t m, int x, int y,
                                             int z, int xm, int xp, int zm, int zp, long long idx,
                                             typename Store<P>::C delta, typename Store<P>::C ule,
                                             typename Store<P>::C (&n)[19]) {
    pull_one<P, p>(v, fin, plb, pr, m, x, y, z, xm, xp, zm, zp, idx, delta, ule, n);
    PullAll<P, p + 1>::run(v, fin, plb, pr, m, x, y, z, xm, xp, zm, zp, idx, delta, ule, n);
  }
};
template <int P>
struct PullAll<P, 19> {
  __device__ __forceinline__ static void run(const View&, const typename Store<P>::T* __restrict__,
                                             const typename Store<P>::C* __restrict__,
                                             const Proto* __restrict__, uint32_t, int, int, int, int,
                                             int, int, int, long long, typename Store<P>::C,
                                             typename Store<P>::C, typename Store<P>::C (&)[19]) {}
};

template <int P>
__global__ void __launch_bounds__(256) k_collide_stream(View v, const typename Store<P>::T* __restrict__ fin,
                                                        typename Store<P>::T* __restrict__ fout) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  __shared__ TC red[32 * 6];
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  TC acc[6] = {0, 0, 0, 0, 0, 0};
  if (idx < v.ncell) {
    const uint32_t m = v.mask[idx];
    if (!(m & 1u)) {
      const int nx = v.nx;
      const int x = (int)(idx % nx);
      const long long t1 = idx / nx;
      const int y = (int)(t1 % v.ny);
      const int z = (int)(t1 / v.ny);
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
      const int zm = z == 0 ? v.nz - 1 : z - 1, zp = z == v.nz - 1 ? 0 : z + 1;
      const Proto* pr = v.proto;
      const TC delta = sel<TC>(pr->delta, pr->delta_f), ule = sel<TC>(pr->ule, pr->ule_f);
      const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
      const TC* plb = reinterpret_cast<const TC*>(v.plb);
      TC n[19];
      n[0] = S::load(fin, idx, (TC)D3Q19::w(0) * rho0, (TC)v.inv_scale);
      PullAll<P, 1>::run(v, fin, plb, pr, m, x, y, z, xm, xp, zm, zp, idx, delta, ule, n);
      TC rho = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const TC cxq = (TC)D3Q19::cx(q), cyq = (TC)D3Q19::cy(q), czq = (TC)D3Q19::cz(q);
        rho += n[q];
        jx += n[q] * cxq; jy += n[q] * cyq; jz += n[q] * czq;
        pxx += n[q] * cxq * cxq; pyy += n[q] * cyq * cyq; pzz += n[q] * czq * czq;
        pxy += n[q] * cxq * cyq; pxz += n[q] * cxq * czq; pyz += n[q] * cyq * czq;
      }
      if (!(rho > (TC)0)) atomicOr(v.err, ERR_UNSTABLE);
      const TC inv = (TC)1 / rho;
      const TC omega = sel<TC>(v.omega_d, v.omega_f);
      const TC gx = sel<TC>(v.g[0], v.g_f[0]), gy = sel<TC>(v.g[1], v.g_f[1]),
               gz = sel<TC>(v.g[2], v.g_f[2]);
      const long long nc = v.ncell;
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const TC fe = feq<TC>(q, rho, jx, jy, jz, inv);
        const TC gc = gx * (TC)D3Q19::cx(q) + gy * (TC)D3Q19::cy(q) + gz * (TC)D3Q19::cz(q);
        const TC o = n[q] - omega * (n[q] - fe) + (TC)3 * (TC)D3Q19::w(q) * gc;
        fout[(long long)q * nc + idx] = S::enc(o, (TC)D3Q19::w(q) * rho0, (TC)v.scale);
      }
      const TC vf = sel<TC>(v.vf_d, v.vf_f);
      const TC third = rho / (TC)3;
      acc[0] = vf * (pxx - jx * jx * inv - third);
      acc[1] = vf * (pyy - jy * jy * inv - third);
      acc[2] = vf * (pzz - jz * jz * inv - third);
      acc[3] = vf * (pxy - jx * jy * inv);
      acc[4] = vf * (pxz - jx * jz * inv);
      acc[5] = vf * (pyz - jy * jz * inv);
    }
  }
  block_sum<TC, 6>(acc, red);
  if (threadIdx.x == 0) {
    double* out = v.visc_part + 6LL * blockIdx.x;
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k] = (double)acc[k];
  }
}

// Moments (rho, j) of the two Lees-Edwards boundary planes, read by the
// crossing pulls of the same step: plane 0 is y = 0, plane 1 is y = ny-1.
template <int P>
__global__ void k_plane_moments(View v, const typename Store<P>::T* __restrict__ fin) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  const long long per = (long long)v.nx * v.nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * per) return;
  const int plane = (int)(t / per);
  const long long r = t % per;
  const int x = (int)(r % v.nx), z = (int)(r / v.nx);
  const int y = plane ? v.ny - 1 : 0;
  const long long idx = x + (long long)v.nx * (y + (long long)v.ny * z);
  TC rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    const TC f = S::load(fin, (long long)q * v.ncell + idx, (TC)D3Q19::w(q) * sel<TC>(v.rho0, v.rho0_f),
                         (TC)v.inv_scale);
    rho += f;
    jx += f * (TC)D3Q19::cx(q); jy += f * (TC)D3Q19::cy(q); jz += f * (TC)D3Q19::cz(q);
  }
  TC* pm = reinterpret_cast<TC*>(v.plane_mom) + 4 * (plane * per + r);
  pm[0] = rho; pm[1] = jx; pm[2] = jy; pm[3] = jz;
}

}  // namespace susp_dev

using namespace susp_dev;

int lb_blocks(long long ncell) { return (int)((ncell + 255) / 256); }

void launch_plane_moments(int prec, const View& v, const void* fin, cudaStream_t s) {
  const long long per = 2LL * v.nx * v.nz;
  const int pb = (int)((per + 255) / 256);
  switch (prec) {
    case 0: k_plane_moments<0><<<pb, 256, 0, s>>>(v, (const double*)fin); break;
    case 1: k_plane_moments<1><<<pb, 256, 0, s>>>(v, (const float*)fin); break;
    case 2: k_plane_moments<2><<<pb, 256, 0, s>>>(v, (const __half*)fin); break;
    default: k_plane_moments<3><<<pb, 256, 0, s>>>(v, (const __nv_bfloat16*)fin); break;
  }
}

void launch_collide_stream(int prec, const View& v, const void* fin, void* fout, cudaStream_t s) {
  const int nb = lb_blocks(v.ncell);
  switch (prec) {
    case 0: k_collide_stream<0><<<nb, 256, 0, s>>>(v, (const double*)fin, (double*)fout); break;
    case 1: k_collide_stream<1><<<nb, 256, 0, s>>>(v, (const float*)fin, (float*)fout); break;
    case 2: k_collide_stream<2><<<nb, 256, 0, s>>>(v, (const __half*)fin, (__half*)fout); break;
    default:
      k_collide_stream<3><<<nb, 256, 0, s>>>(v, (const __nv_bfloat16*)fin, (__nv_bfloat16*)fout);
      break;
  }
}
