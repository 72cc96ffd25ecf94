// lbm.cu — fused D3Q19 collide-stream kernel (pull scheme, A/B buffers).
//
// Per fluid node r and direction p the post-streaming population is
//   n_p(r, t+1) = n*_p(r - c_p, t)                          (Eq. 3, pull form)
// with two exceptions:
//   * the source r - c_p = s is solid: moving bounce-back (Eq. 7, 8)
//       n_p(r, t+1) = n*_q(r, t) - 6 C^q rho0 (u_b . c_q),  q = -p,
//       u_b = U + Omega x (r_b - R), r_b = r + c_q / 2.
//     The boundary-link kernel, which runs after the node map is updated,
//     stores this value in the slot p of s (each such slot has exactly one
//     receiver), so the pull reads it like any other population;
//   * the source lies beyond a Lees-Edwards plane (y = 0 from below or
//     y = ny-1 from above): the image box is shifted by -/+ Delta in x and
//     moves with -/+ U_LE, so the value is linearly interpolated between the
//     two nodes straddling x - c_px +/- Delta on the opposite plane and
//     Galilean-shifted by n^eq(rho, j -/+ rho U_LE e_x) - n^eq(rho, j);
//     the nearer of the two nodes decides solid (bounce-back, evaluated
//     here) or fluid, and a solid farther node leaves the nearer one alone
//     as the source.
// Solid nodes store the rest state (their slots are rewritten by the link
// kernel where a receiver needs them).  Then the BGK collision (Eq. 4, 5
// with every non-conserved mode relaxed by 1/tau) and an optional uniform
// body force 3 C^q (g . c_q).  Each block also sums the viscous stress
// -(1 - 1/(2 tau)) Pi^neq of its fluid nodes.
//
// Bytes per fluid node and step: 19 loads + 19 stores of the storage type
// plus the 4-byte owner word (algorithmic 2 * 19 * s).
#include <cuda.h>

#include <mutex>

#include "susp_dev.cuh"

namespace susp_dev {

// Moving-wall term of Eq. 7 for the population p pulled at node (x, y, z)
// from the solid node r - c_p of particle i:  -6 C^q rho0 (u_b . c_q) with
// q = -p, u_b = U + Omega x (r_b - R) at r_b = r + c_q / 2 (Eq. 8).
template <typename TC>
__device__ __forceinline__ TC wall_term(const View& v, const TC* __restrict__ plb, int i, int x, int y,
                                        int z, int q, TC delta, TC ule, TC rho0) {
  const TC* pp = plb + 12 * i;
  const TC cqx = (TC)D3Q19::cx(q), cqy = (TC)D3Q19::cy(q), cqz = (TC)D3Q19::cz(q);
  TC dx = (TC)x + (TC)0.5 * cqx - pp[0];
  TC dy = (TC)y + (TC)0.5 * cqy - pp[1];
  TC dz = (TC)z + (TC)0.5 * cqz - pp[2];
  const int k = le_image_v(v, dx, dy, dz, delta);
  const TC ubx = pp[3] + (pp[7] * dz - pp[8] * dy) + (TC)k * ule;
  const TC uby = pp[4] + (pp[8] * dx - pp[6] * dz);
  const TC ubz = pp[5] + (pp[6] * dy - pp[7] * dx);
  const TC cu = ubx * cqx + uby * cqy + ubz * cqz;
  return -(TC)6 * wq<TC>(q) * rho0 * cu;
}

// Pull across a Lees-Edwards plane (direction p with c_py = +1 at y = 0, or
// c_py = -1 at y = ny-1).
template <int P, int p>
__device__ __forceinline__ typename Store<P>::C le_pull(const View& v, const typename Store<P>::T* __restrict__ fin,
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
    const TC self = S::load(fin, (long long)q * nc + idx, base_q, (TC)v.inv_scale);
    return self + wall_term<TC>(v, plb, on, x, y, z, q, delta, ule, rho0);
  }
  const TC* pm = reinterpret_cast<const TC*>(pm_in_of(v)) + (below ? 4LL * v.nz * nx : 0);
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

// Plain pull of population p from r - c_p (32-bit node offsets: interior
// offsets are fixed sums of the precomputed x / z wrap deltas and -c_py nx).
// Where r - c_p is solid the slot holds the bounce-back value.
template <int P, int p, bool BND>
__device__ __forceinline__ void pull_one(const View& v, const typename Store<P>::T* __restrict__ fin,
                                         const typename Store<P>::C* __restrict__ plb,
                                         const Proto* __restrict__ pr, int x, int y, int z, int idx,
                                         int dxm, int dxp, int dzm, int dzp,
                                         typename Store<P>::C rho0, typename Store<P>::C (&n)[19]) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  constexpr int cpx = D3Q19::cx(p), cpy = D3Q19::cy(p), cpz = D3Q19::cz(p);
  const int sy = y - cpy;
  if (BND && cpy != 0 && (sy < 0 || sy >= v.ny)) {
    n[p] = le_pull<P, p>(v, fin, plb, pr, x, y, z, idx);
    return;
  }
  const int off = (cpx == 1 ? dxm : (cpx == -1 ? dxp : 0)) - cpy * v.nx + (cpz == 1 ? dzm : (cpz == -1 ? dzp : 0));
  // element index in 32 bits: 19 * ncell < 2^32 for every accepted box
  const uint32_t e = (uint32_t)p * (uint32_t)v.ncell + (uint32_t)(idx + off);
  n[p] = S::load(fin, e, (TC)D3Q19::w(p) * rho0, (TC)v.inv_scale);
}

template <int P, int p, bool BND>
struct PullAll {
  __device__ __forceinline__ static void run(const View& v, const typename Store<P>::T* __restrict__ fin,
                                             const typename Store<P>::C* __restrict__ plb,
                                             const Proto* __restrict__ pr, int x, int y, int z, int idx,
                                             int dxm, int dxp, int dzm, int dzp,
                                             typename Store<P>::C rho0, typename Store<P>::C (&n)[19]) {
    pull_one<P, p, BND>(v, fin, plb, pr, x, y, z, idx, dxm, dxp, dzm, dzp, rho0, n);
    PullAll<P, p + 1, BND>::run(v, fin, plb, pr, x, y, z, idx, dxm, dxp, dzm, dzp, rho0, n);
  }
};
template <int P, bool BND>
struct PullAll<P, 19, BND> {
  __device__ __forceinline__ static void run(const View&, const typename Store<P>::T* __restrict__,
                                             const typename Store<P>::C* __restrict__,
                                             const Proto* __restrict__, int, int, int, int, int, int,
                                             int, int, typename Store<P>::C, typename Store<P>::C (&)[19]) {}
};

template <int P>
__device__ __forceinline__ void lb_collide(const View& v, typename Store<P>::T* __restrict__ fout, int idx,
                                           typename Store<P>::C (&n)[19], typename Store<P>::C (&acc)[6],
                                           typename Store<P>::C* __restrict__ pmo);

// One lattice node: pull (Eq. 3; bounce-back values sit in the solid
// sources' slots) with the Lees-Edwards planes, BGK collision (Eq. 4, 5),
// store, viscous-stress accumulation.  BND: the node lies on a Lees-Edwards
// plane (y = 0 or ny-1); interior rows compile without the plane code.
template <int P, bool BND>
__device__ __forceinline__ void lb_node(const View& v, const typename Store<P>::T* __restrict__ fin,
                                        typename Store<P>::T* __restrict__ fout, int x, int y, int z,
                                        int dzm, int dzp, typename Store<P>::C (&acc)[6]) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  const int nx = v.nx;
  const int idx = x + nx * (y + v.ny * z);
  const uint32_t nc = (uint32_t)v.ncell;   // 19 * ncell < 2^32 for every accepted box
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
  if (v.owner[idx] >= 0) {
    // solid node: its populations are undefined; writing the rest state keeps
    // every stored sector complete (no read-for-ownership of partial sectors)
#pragma unroll
    for (int q = 0; q < 19; ++q)
      fout[(uint32_t)q * nc + (uint32_t)idx] = S::enc((TC)D3Q19::w(q) * rho0, (TC)D3Q19::w(q) * rho0, (TC)v.scale);
    return;
  }
  const int dxm = x == 0 ? nx - 1 : -1, dxp = x == nx - 1 ? 1 - nx : 1;
  const Proto* pr = v.proto;
  const TC* plb = reinterpret_cast<const TC*>(v.plb);
  TC n[19];
  n[0] = S::load(fin, (uint32_t)idx, (TC)D3Q19::w(0) * rho0, (TC)v.inv_scale);
  PullAll<P, 1, BND>::run(v, fin, plb, pr, x, y, z, idx, dxm, dxp, dzm, dzp, rho0, n);
  // a node on a Lees-Edwards plane also writes the moments of its new
  // populations, which the next step's crossing pulls read
  TC* pmo = nullptr;
  if (BND) pmo = reinterpret_cast<TC*>(pm_out_of(v)) + 4LL * ((y == 0 ? 0 : (long long)v.nz * nx) + x + (long long)nx * z);
  lb_collide<P>(v, fout, idx, n, acc, pmo);
}

// Collision (Eq. 4, 5: BGK, or Ladd's linear operator when the box asks for
// it) of one fluid node from its pulled populations n, optional body force,
// store, viscous-stress accumulation.
template <int P>
__device__ __forceinline__ void lb_collide(const View& v, typename Store<P>::T* __restrict__ fout, int idx,
                                           typename Store<P>::C (&n)[19], typename Store<P>::C (&acc)[6],
                                           typename Store<P>::C* __restrict__ pmo) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  const uint32_t nc = (uint32_t)v.ncell;
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
  // moments from the opposite pairs (q, q+1), q odd: sums s and differences d
  TC sp[9], dp[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) { sp[k] = n[2 * k + 1] + n[2 * k + 2]; dp[k] = n[2 * k + 1] - n[2 * k + 2]; }
  // second moments: for FP32 arithmetic from the deviations n - C^q rho0
  // (exact differences), so that Pi - rho I / 3 does not cancel two values of
  // size 1/3; rsec is then rho - rho0 instead of rho
  TC ss[9], rsec;
  if constexpr (P == 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) ss[k] = sp[k];
    rsec = n[0];
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const TC wr = (TC)D3Q19::w(2 * k + 1) * rho0;
      ss[k] = (n[2 * k + 1] - wr) + (n[2 * k + 2] - wr);
    }
    rsec = n[0] - (TC)D3Q19::w(0) * rho0;
  }
  TC rho = n[0], jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int q = 2 * k + 1;
    const int cxq = D3Q19::cx(q), cyq = D3Q19::cy(q), czq = D3Q19::cz(q);
    rho += sp[k];
    rsec += ss[k];
    if (cxq) jx += cxq > 0 ? dp[k] : -dp[k];
    if (cyq) jy += cyq > 0 ? dp[k] : -dp[k];
    if (czq) jz += czq > 0 ? dp[k] : -dp[k];
    if (cxq) pxx += ss[k];
    if (cyq) pyy += ss[k];
    if (czq) pzz += ss[k];
    if (cxq && cyq) pxy += cxq * cyq > 0 ? ss[k] : -ss[k];
    if (cxq && czq) pxz += cxq * czq > 0 ? ss[k] : -ss[k];
    if (cyq && czq) pyz += cyq * czq > 0 ? ss[k] : -ss[k];
  }
  if (!(rho > (TC)0)) atomicOr(v.err, ERR_UNSTABLE);
  const TC inv = (TC)1 / rho;
  const TC omega = sel<TC>(v.omega_d, v.omega_f);
  const TC jj = jx * jx + jy * jy + jz * jz;
  // n^eq_q = C^q [rho + 3 j.c + 4.5 (j.c)^2 / rho - 1.5 j^2 / rho]; for an
  // opposite pair the first, third and fourth terms are shared
  const TC base = rho - (TC)1.5 * jj * inv;
  const TC g0 = sel<TC>(v.g[0], v.g_f[0]), g1 = sel<TC>(v.g[1], v.g_f[1]), g2 = sel<TC>(v.g[2], v.g_f[2]);
  const bool hg = v.has_g != 0;
  if (v.ladd) {
    // Ladd's linear operator (Eq. 5 by its eigenvalues):
    //   n*_q = n^eq_q + (9/2) C^q Pi*:(c_q c_q - I/3),
    //   Pi* = (1 + lambda) bar(Pi^neq) + (1 + lambda_v) tr(Pi^neq) I / 3,
    // the ghost modes removed; viscous stress -(1 + lambda/2) of the
    // traceless and -(1 + lambda_v/2) of the isotropic non-equilibrium stress
    const TC third = rsec / (TC)3;
    const TC nxx = pxx - jx * jx * inv - third, nyy = pyy - jy * jy * inv - third, nzz = pzz - jz * jz * inv - third;
    const TC nxy = pxy - jx * jy * inv, nxz = pxz - jx * jz * inv, nyz = pyz - jy * jz * inv;
    const TC ls = sel<TC>(v.ls_d, v.ls_f), lb = sel<TC>(v.lb_d, v.lb_f);
    const TC t3 = (nxx + nyy + nzz) / (TC)3;
    const TC sxx = ls * (nxx - t3) + lb * t3, syy = ls * (nyy - t3) + lb * t3, szz = ls * (nzz - t3) + lb * t3;
    const TC sxy = ls * nxy, sxz = ls * nxz, syz = ls * nyz;
    const TC st3 = (sxx + syy + szz) / (TC)3;
    TC mr, mjx = 0, mjy = 0, mjz = 0;   // moments of the new populations
    {
      const TC w0 = (TC)D3Q19::w(0);
      const TC o0 = w0 * base - (TC)4.5 * w0 * st3;
      fout[idx] = S::enc(o0, w0 * rho0, (TC)v.scale);
      mr = o0;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int q = 2 * k + 1;
      const int cxq = D3Q19::cx(q), cyq = D3Q19::cy(q), czq = D3Q19::cz(q);
      TC jc = 0, ccp = 0;
      if (cxq) { jc += cxq > 0 ? jx : -jx; ccp += sxx; }
      if (cyq) { jc += cyq > 0 ? jy : -jy; ccp += syy; }
      if (czq) { jc += czq > 0 ? jz : -jz; ccp += szz; }
      if (cxq && cyq) ccp += (TC)2 * (cxq * cyq > 0 ? sxy : -sxy);
      if (cxq && czq) ccp += (TC)2 * (cxq * czq > 0 ? sxz : -sxz);
      if (cyq && czq) ccp += (TC)2 * (cyq * czq > 0 ? syz : -syz);
      const TC w = (TC)D3Q19::w(q);
      const TC sym = w * (base + (TC)4.5 * jc * jc * inv) + (TC)4.5 * w * (ccp - st3);
      const TC anti = (TC)3 * w * jc;
      TC oq = sym + anti, oo = sym - anti;
      if (hg) {
        TC gc = 0;
        if (cxq) gc += cxq > 0 ? g0 : -g0;
        if (cyq) gc += cyq > 0 ? g1 : -g1;
        if (czq) gc += czq > 0 ? g2 : -g2;
        const TC gq = (TC)3 * w * gc;
        oq += gq;
        oo -= gq;
      }
      fout[(uint32_t)q * nc + (uint32_t)idx] = S::enc(oq, w * rho0, (TC)v.scale);
      fout[(uint32_t)(q + 1) * nc + (uint32_t)idx] = S::enc(oo, w * rho0, (TC)v.scale);
      mr += oq + oo;
      if (cxq) mjx += cxq > 0 ? oq - oo : oo - oq;
      if (cyq) mjy += cyq > 0 ? oq - oo : oo - oq;
      if (czq) mjz += czq > 0 ? oq - oo : oo - oq;
    }
    if (pmo) { pmo[0] = mr; pmo[1] = mjx; pmo[2] = mjy; pmo[3] = mjz; }
    const TC vf = sel<TC>(v.vf_d, v.vf_f), vfb = sel<TC>(v.vfb_d, v.vfb_f);
    acc[0] += vf * (nxx - t3) + vfb * t3;
    acc[1] += vf * (nyy - t3) + vfb * t3;
    acc[2] += vf * (nzz - t3) + vfb * t3;
    acc[3] += vf * nxy;
    acc[4] += vf * nxz;
    acc[5] += vf * nyz;
    return;
  }
  TC mr, mjx = 0, mjy = 0, mjz = 0;   // moments of the new populations
  {
    const TC fe = (TC)D3Q19::w(0) * base;
    const TC o = n[0] + omega * (fe - n[0]);
    fout[idx] = S::enc(o, (TC)D3Q19::w(0) * rho0, (TC)v.scale);
    mr = o;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int q = 2 * k + 1;
    const int cxq = D3Q19::cx(q), cyq = D3Q19::cy(q), czq = D3Q19::cz(q);
    TC jc = 0;
    if (cxq) jc += cxq > 0 ? jx : -jx;
    if (cyq) jc += cyq > 0 ? jy : -jy;
    if (czq) jc += czq > 0 ? jz : -jz;
    const TC w = (TC)D3Q19::w(q);
    const TC sym = w * (base + (TC)4.5 * jc * jc * inv);
    TC anti = (TC)3 * w * jc;
    TC oq = n[q] + omega * (sym + anti - n[q]);
    TC oo = n[q + 1] + omega * (sym - anti - n[q + 1]);
    if (hg) {
      TC gc = 0;
      if (cxq) gc += cxq > 0 ? g0 : -g0;
      if (cyq) gc += cyq > 0 ? g1 : -g1;
      if (czq) gc += czq > 0 ? g2 : -g2;
      const TC gq = (TC)3 * w * gc;
      oq += gq;
      oo -= gq;
    }
    fout[(uint32_t)q * nc + (uint32_t)idx] = S::enc(oq, w * rho0, (TC)v.scale);
    fout[(uint32_t)(q + 1) * nc + (uint32_t)idx] = S::enc(oo, w * rho0, (TC)v.scale);
    mr += oq + oo;
    if (cxq) mjx += cxq > 0 ? oq - oo : oo - oq;
    if (cyq) mjy += cyq > 0 ? oq - oo : oo - oq;
    if (czq) mjz += czq > 0 ? oq - oo : oo - oq;
  }
  if (pmo) { pmo[0] = mr; pmo[1] = mjx; pmo[2] = mjy; pmo[3] = mjz; }
  const TC vf = sel<TC>(v.vf_d, v.vf_f);
  const TC third = rsec / (TC)3;
  acc[0] += vf * (pxx - jx * jx * inv - third);
  acc[1] += vf * (pyy - jy * jy * inv - third);
  acc[2] += vf * (pzz - jz * jz * inv - third);
  acc[3] += vf * (pxy - jx * jy * inv);
  acc[4] += vf * (pxz - jx * jz * inv);
  acc[5] += vf * (pyz - jy * jz * inv);
}

// ---------------------------------------------------------------------------
// Row pairs (FP32 compute over FP32, FP16 or BF16 storage).  A lane takes the
// node (x, y, z) and the node above it, (x, y + 1, z), both off the
// Lees-Edwards planes, and carries the two through the same arithmetic with
// the packed FP32x2 instructions of sm_100+ (one instruction per operation
// for both nodes, each an ordinary FP32 rounding).  The collision runs on
// deviations from the rest state, u = s (n - C^q rho0) with the storage's
// scale s (1 for FP32 and BF16): the deviation storages hold u itself, and
// FP32 storage subtracts C^q rho0 on load (exact, the two are within a factor
// of two) and adds it back through the stored constants.  The moments of the
// deviations carry no cancellation against the rest state (Pi_xx - rho / 3 is
// formed from values of size n^neq, not of size 1/3).  With R = sum_q u_q,
// J = sum_q u_q c_q and iota = 1 / (R + s rho0) = 1 / (s rho):
//   u^eq_q = C^q [R + 3 J.c_q + (4.5 (J.c_q)^2 - 1.5 J.J) iota],
//   u*_q   = u_q + omega (u^eq_q - u_q),
// which is n^eq of Eq. 4 and the BGK relaxation of Eq. 5 in those units; the
// viscous stress -(1 - 1/(2 tau)) Pi^neq is (Pi_u - J J iota - R I / 3) times
// the same factor and 1 / s.  A solid node loads nothing (its loads are
// predicated off, so it reads no memory; its deviations are zero) and stores
// the rest state, which nothing reads: the link kernel rewrites every slot
// that a receiver pulls.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_s(float a) { return make_float2(a, a); }

template <int P> struct Raw;
template <> struct Raw<1> {
  __device__ static float ld(const float* f, uint32_t e) { return __ldg(f + e); }
  __device__ static void st(float* f, uint32_t e, float u) { f[e] = u; }
};
template <> struct Raw<2> {
  __device__ static float ld(const __half* f, uint32_t e) { return __half2float(__ldg(f + e)); }
  __device__ static void st(__half* f, uint32_t e, float u) { f[e] = __float2half_rn(u); }
};
template <> struct Raw<3> {
  __device__ static float ld(const __nv_bfloat16* f, uint32_t e) { return __bfloat162float(__ldg(f + e)); }
  __device__ static void st(__nv_bfloat16* f, uint32_t e, float u) { f[e] = __float2bfloat16_rn(u); }
};

// +c or -c of a packed pair by the sign of a lattice component (0: nothing).
template <int c>
__device__ __forceinline__ float2 p_acc(float2 acc, float2 v) {
  if constexpr (c > 0) return p_add(acc, v);
  else if constexpr (c < 0) return p_sub(acc, v);
  else return acc;
}

template <int P, int p>
struct PairPull {
  __device__ __forceinline__ static void run(const typename Store<P>::T* __restrict__ fin, uint32_t nc, int nx,
                                             uint32_t iA, int dxm, int dxp, int dzm, int dzp, bool fA, bool fB,
                                             float rest, float2 (&u)[19]) {
    constexpr int cpx = D3Q19::cx(p), cpy = D3Q19::cy(p), cpz = D3Q19::cz(p);
    const int off = (cpx == 1 ? dxm : (cpx == -1 ? dxp : 0)) - cpy * nx + (cpz == 1 ? dzm : (cpz == -1 ? dzp : 0));
    const uint32_t e = (uint32_t)p * nc + iA + (uint32_t)off;
    // FP32 storage holds n: its deviation from C^q rho0 (rho0 = rest / C^0)
    const float r = (P == 1) ? (float)D3Q19::w(p) * rest : 0.0f;
    u[p].x = fA ? Raw<P>::ld(fin, e) - r : 0.0f;
    u[p].y = fB ? Raw<P>::ld(fin, e + (uint32_t)nx) - r : 0.0f;
    PairPull<P, p + 1>::run(fin, nc, nx, iA, dxm, dxp, dzm, dzp, fA, fB, rest, u);
  }
};
template <int P>
struct PairPull<P, 19> {
  __device__ __forceinline__ static void run(const typename Store<P>::T* __restrict__, uint32_t, int, uint32_t,
                                             int, int, int, int, bool, bool, float, float2 (&)[19]) {}
};

// Collision of the opposite pair (q, q + 1), q = 2k + 1, and its stores.
// Relaxed non-equilibrium stress of Ladd's operator (storage units), per node
// of the pair: Pi* = (1 + lambda) bar(Pi^neq) + (1 + lambda_v) tr(Pi^neq) I / 3
// and st3 = tr(Pi*) / 3.
struct PairPi {
  float2 xx, yy, zz, xy, xz, yz, st3;
};

template <int P, int k, bool L>
struct PairCollide {
  __device__ __forceinline__ static void run(typename Store<P>::T* __restrict__ fout, uint32_t nc, uint32_t iA,
                                             int nx, const float2 (&u)[19], float2 jx, float2 jy, float2 jz,
                                             float2 omc, float2 a1, float2 b1, float2 a2, float2 b2, float c1,
                                             float c2, bool hg, float g0, float g1, float g2, const PairPi& pi) {
    constexpr int q = 2 * k + 1;
    constexpr int cx = D3Q19::cx(q), cy = D3Q19::cy(q), cz = D3Q19::cz(q);
    constexpr bool first = (q <= 6);   // C^q = 1/18, else 1/36
    float2 jc = make_float2(0.0f, 0.0f);
    if constexpr (cx != 0 && cy == 0 && cz == 0) jc = cx > 0 ? jx : p_sub(jc, jx);
    else if constexpr (cx == 0 && cy != 0 && cz == 0) jc = cy > 0 ? jy : p_sub(jc, jy);
    else if constexpr (cx == 0 && cy == 0 && cz != 0) jc = cz > 0 ? jz : p_sub(jc, jz);
    else {
      jc = p_acc<cx>(jc, jx);
      jc = p_acc<cy>(jc, jy);
      jc = p_acc<cz>(jc, jz);
    }
    const float2 sym = p_fma(p_mul(jc, jc), first ? b1 : b2, first ? a1 : a2);
    const float2 anti = p_mul(jc, p_s(first ? c1 : c2));
    float2 plus = p_add(sym, anti), minus = p_sub(sym, anti);
    if constexpr (L) {
      // Ladd: + (9/2) C^q Pi*:(c_q c_q - I/3), the same for q and -q
      float2 ccp = make_float2(0.0f, 0.0f);
      if constexpr (cx != 0) ccp = p_add(ccp, pi.xx);
      if constexpr (cy != 0) ccp = p_add(ccp, pi.yy);
      if constexpr (cz != 0) ccp = p_add(ccp, pi.zz);
      if constexpr (cx != 0 && cy != 0) ccp = p_fma(p_s(2.0f * cx * cy), pi.xy, ccp);
      if constexpr (cx != 0 && cz != 0) ccp = p_fma(p_s(2.0f * cx * cz), pi.xz, ccp);
      if constexpr (cy != 0 && cz != 0) ccp = p_fma(p_s(2.0f * cy * cz), pi.yz, ccp);
      const float2 e = p_mul(p_s(4.5f * (first ? 1.0f / 18.0f : 1.0f / 36.0f)), p_sub(ccp, pi.st3));
      plus = p_add(plus, e);
      minus = p_add(minus, e);
    }
    if (hg) {
      // body force 3 C^q (g . c_q) (g given in storage units times 3)
      float gc = 0.0f;
      if constexpr (cx != 0) gc += cx > 0 ? g0 : -g0;
      if constexpr (cy != 0) gc += cy > 0 ? g1 : -g1;
      if constexpr (cz != 0) gc += cz > 0 ? g2 : -g2;
      const float gq = (first ? 1.0f / 18.0f : 1.0f / 36.0f) * gc;
      plus = p_add(plus, p_s(gq));
      minus = p_sub(minus, p_s(gq));
    }
    const float2 oq = p_fma(omc, u[q], plus);
    const float2 oo = p_fma(omc, u[q + 1], minus);
    const uint32_t eq = (uint32_t)q * nc + iA, eo = (uint32_t)(q + 1) * nc + iA;
    Raw<P>::st(fout, eq, oq.x);
    Raw<P>::st(fout, eq + (uint32_t)nx, oq.y);
    Raw<P>::st(fout, eo, oo.x);
    Raw<P>::st(fout, eo + (uint32_t)nx, oo.y);
    PairCollide<P, k + 1, L>::run(fout, nc, iA, nx, u, jx, jy, jz, omc, a1, b1, a2, b2, c1, c2, hg, g0, g1, g2, pi);
  }
};
template <int P, bool L>
struct PairCollide<P, 9, L> {
  __device__ __forceinline__ static void run(typename Store<P>::T* __restrict__, uint32_t, uint32_t, int,
                                             const float2 (&)[19], float2, float2, float2, float2, float2, float2,
                                             float2, float2, float, float, bool, float, float, float,
                                             const PairPi&) {}
};

// Moments of the packed pulled values: R, J and the second moments Pi_u.
template <int k>
__device__ __forceinline__ void pair_moments(const float2 (&u)[19], float2& R, float2& jx, float2& jy, float2& jz,
                                             float2& pxx, float2& pyy, float2& pzz, float2& pxy, float2& pxz,
                                             float2& pyz) {
  if constexpr (k < 9) {
    constexpr int q = 2 * k + 1;
    constexpr int cx = D3Q19::cx(q), cy = D3Q19::cy(q), cz = D3Q19::cz(q);
    const float2 sp = p_add(u[q], u[q + 1]), dp = p_sub(u[q], u[q + 1]);
    R = p_add(R, sp);
    jx = p_acc<cx>(jx, dp);
    jy = p_acc<cy>(jy, dp);
    jz = p_acc<cz>(jz, dp);
    if constexpr (cx != 0) pxx = p_add(pxx, sp);
    if constexpr (cy != 0) pyy = p_add(pyy, sp);
    if constexpr (cz != 0) pzz = p_add(pzz, sp);
    if constexpr (cx != 0 && cy != 0) pxy = p_acc<cx * cy>(pxy, sp);
    if constexpr (cx != 0 && cz != 0) pxz = p_acc<cx * cz>(pxz, sp);
    if constexpr (cy != 0 && cz != 0) pyz = p_acc<cy * cz>(pyz, sp);
    pair_moments<k + 1>(u, R, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz);
  }
}

// Collision of a row pair from its pulled deviations u (zero for a solid
// node), stores and viscous-stress sums (packed: acc2[k].x and .y for the
// two nodes).  L: Ladd's linear operator, which is the BGK form at
// omega = 1 plus the relaxed stress term (9/2) C^q Pi*:(c_q c_q - I/3); its
// viscous stress -(1 + lambda/2) bar(Pi^neq) - (1 + lambda_v/2) tr I / 3 is
// summed as bar(Pi^neq) + (vfb / vf) tr I / 3, times vf at the end.
template <int P, bool L>
__device__ __forceinline__ void pair_collide(const View& v, typename Store<P>::T* __restrict__ fout, uint32_t iA,
                                             bool fA, bool fB, float2 (&u)[19], float2 (&acc2)[6]) {
  const int nx = v.nx;
  const uint32_t nc = (uint32_t)v.ncell;
  const float rho0 = v.rho0_f;
  const float2 zero = make_float2(0.0f, 0.0f);
  float2 R = u[0], jx = zero, jy = zero, jz = zero, pxx = zero, pyy = zero, pzz = zero, pxy = zero,
         pxz = zero, pyz = zero;
  pair_moments<0>(u, R, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz);
  // R + s rho0 is s rho
  const float su = (P == 2) ? v.scale : 1.0f;
  const float2 rs = p_add(R, p_s(su * rho0));
  if ((fA && !(rs.x > 0.0f)) || (fB && !(rs.y > 0.0f))) atomicOr(v.err, ERR_UNSTABLE);
  const float2 iota = make_float2(__fdividef(1.0f, rs.x), __fdividef(1.0f, rs.y));
  const float2 jj = p_fma(jz, jz, p_fma(jy, jy, p_mul(jx, jx)));
  const float2 base = p_fma(p_s(-1.5f), p_mul(jj, iota), R);
  const float om = L ? 1.0f : v.omega_f;
  const float2 omc = p_s(1.0f - om);
  constexpr float w0 = 1.0f / 3.0f, w1 = 1.0f / 18.0f, w2 = 1.0f / 36.0f;
  // non-equilibrium stress Pi_u - J J iota - R I / 3 (Ladd needs it before
  // the collision, BGK only for the viscous sums)
  const float2 r3 = p_mul(R, p_s(1.0f / 3.0f));
  const float2 jxi = p_mul(jx, iota), jyi = p_mul(jy, iota);
  PairPi pi;
  float2 nxx, nyy, nzz, nxy, nxz, nyz, t3;
  if constexpr (L) {
    nxx = p_sub(p_sub(pxx, p_mul(jx, jxi)), r3);
    nyy = p_sub(p_sub(pyy, p_mul(jy, jyi)), r3);
    nzz = p_sub(p_sub(pzz, p_mul(jz, p_mul(jz, iota))), r3);
    nxy = p_sub(pxy, p_mul(jy, jxi));
    nxz = p_sub(pxz, p_mul(jz, jxi));
    nyz = p_sub(pyz, p_mul(jz, jyi));
    t3 = p_mul(p_add(p_add(nxx, nyy), nzz), p_s(1.0f / 3.0f));
    const float2 ls = p_s(v.ls_f), lbt = p_mul(p_s(v.lb_f), t3);
    pi.xx = p_fma(ls, p_sub(nxx, t3), lbt);
    pi.yy = p_fma(ls, p_sub(nyy, t3), lbt);
    pi.zz = p_fma(ls, p_sub(nzz, t3), lbt);
    pi.xy = p_mul(ls, nxy);
    pi.xz = p_mul(ls, nxz);
    pi.yz = p_mul(ls, nyz);
    pi.st3 = lbt;
  }
  // omega-scaled equilibrium pieces per weight class, with the rest state
  // that FP32 storage adds back
  const float rs0 = (P == 1) ? w0 * rho0 : 0.0f, rs1 = (P == 1) ? w1 * rho0 : 0.0f,
              rs2 = (P == 1) ? w2 * rho0 : 0.0f;
  const float2 a0 = p_fma(base, p_s(om * w0), p_s(rs0));
  const float2 a1 = p_fma(base, p_s(om * w1), p_s(rs1)), a2 = p_fma(base, p_s(om * w2), p_s(rs2));
  const float2 b1 = p_mul(iota, p_s(4.5f * om * w1)), b2 = p_mul(iota, p_s(4.5f * om * w2));
  const float c1 = 3.0f * om * w1, c2 = 3.0f * om * w2;
  float2 o0 = p_fma(omc, u[0], a0);
  if constexpr (L) o0 = p_fma(p_s(-4.5f * w0), pi.st3, o0);   // c_0 = 0: only the -I/3 part
  Raw<P>::st(fout, iA, o0.x);
  Raw<P>::st(fout, iA + (uint32_t)nx, o0.y);
  const float gs = 3.0f * su;
  const bool hg = v.has_g != 0;
  PairCollide<P, 0, L>::run(fout, nc, iA, nx, u, jx, jy, jz, omc, a1, b1, a2, b2, c1, c2, hg, gs * v.g_f[0],
                            gs * v.g_f[1], gs * v.g_f[2], pi);
  // viscous stress of the fluid nodes
  const float2 m = make_float2(fA ? 1.0f : 0.0f, fB ? 1.0f : 0.0f);
  if constexpr (L) {
    const float2 tb = p_mul(p_s(v.vfb_f / v.vf_f - 1.0f), t3);   // trace part with vfb instead of vf
    acc2[0] = p_fma(m, p_add(nxx, tb), acc2[0]);
    acc2[1] = p_fma(m, p_add(nyy, tb), acc2[1]);
    acc2[2] = p_fma(m, p_add(nzz, tb), acc2[2]);
    acc2[3] = p_fma(m, nxy, acc2[3]);
    acc2[4] = p_fma(m, nxz, acc2[4]);
    acc2[5] = p_fma(m, nyz, acc2[5]);
  } else {
    acc2[0] = p_fma(m, p_sub(p_sub(pxx, p_mul(jx, jxi)), r3), acc2[0]);
    acc2[1] = p_fma(m, p_sub(p_sub(pyy, p_mul(jy, jyi)), r3), acc2[1]);
    acc2[2] = p_fma(m, p_sub(p_sub(pzz, p_mul(jz, p_mul(jz, iota))), r3), acc2[2]);
    acc2[3] = p_fma(m, p_sub(pxy, p_mul(jy, jxi)), acc2[3]);
    acc2[4] = p_fma(m, p_sub(pxz, p_mul(jz, jxi)), acc2[4]);
    acc2[5] = p_fma(m, p_sub(pyz, p_mul(jz, jyi)), acc2[5]);
  }
}

// Two interior nodes (x, y, z) and (x, y + 1, z): pulls straight from global
// memory, then the collision above.
template <int P, bool L>
__device__ __forceinline__ void lb_pair(const View& v, const typename Store<P>::T* __restrict__ fin,
                                        typename Store<P>::T* __restrict__ fout, int x, int y, int z, int dzm,
                                        int dzp, float2 (&acc2)[6]) {
  const int nx = v.nx;
  const uint32_t iA = (uint32_t)(x + nx * (y + v.ny * z));
  const uint32_t nc = (uint32_t)v.ncell;   // 19 * ncell < 2^32 for every accepted box
  const bool fA = v.owner[iA] < 0, fB = v.owner[iA + (uint32_t)nx] < 0;
  const int dxm = x == 0 ? nx - 1 : -1, dxp = x == nx - 1 ? 1 - nx : 1;
  float2 u[19];
  PairPull<P, 0>::run(fin, nc, nx, iA, dxm, dxp, dzm, dzp, fA, fB, v.rho0_f, u);
  pair_collide<P, L>(v, fout, iA, fA, fB, u, acc2);
}

// One node of a row that has no interior partner (a Lees-Edwards plane row,
// or the last row of an odd L_y): the scalar path, kept out
// of line so that its registers do not count against the row pairs.
template <int P>
__device__ __noinline__ void lb_node_single(const View& v, const typename Store<P>::T* __restrict__ fin,
                                            typename Store<P>::T* __restrict__ fout, int x, int y, int z, int dzm,
                                            int dzp, float (&acc)[6]) {
  if (y == 0 || y == v.ny - 1) lb_node<P, true>(v, fin, fout, x, y, z, dzm, dzp, acc);
  else lb_node<P, false>(v, fin, fout, x, y, z, dzm, dzp, acc);
}

// Exact division by a runtime divisor d >= 1 for 0 <= n < 2^31 with one
// multiply-high (Granlund and Montgomery, 1994): m = ceil(2^(31 + l) / d),
// l = ceil(log2 d), q = floor(n m / 2^(31 + l)).
struct FastDiv {
  uint32_t m;
  int sh;   // l - 1, or -1 for d = 1
  __device__ void init(uint32_t d) {
    if (d <= 1) { m = 0; sh = -1; return; }
    const int l = 32 - __clz((int)(d - 1));
    m = (uint32_t)(((1ull << (31 + l)) + d - 1) / d);
    sh = l - 1;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return sh < 0 ? n : (__umulhi(n, m) >> sh); }
};

// Persistent grid over the 32 (x) by 2^tile_lg (y) tiles of every box (z slowest
// within a box); each block takes a contiguous range of tiles, sums its nodes'
// viscous stress per box and adds it to the box's accumulator when its range
// leaves the box.  Within a block the warps claim the 32-node rows of the
// range one at a time from a shared counter, so a warp that draws the costly
// Lees-Edwards plane rows does not hold the others at the block's barrier.
template <int P>
__global__ void __launch_bounds__(256) k_collide_stream(Batch B) {
  using TC = typename Store<P>::C;
  using T = typename Store<P>::T;
  __shared__ TC red[32 * 6];
  __shared__ int s_next;
  const int total = B.tile_off[B.nbox];
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  if (t0 >= t1) return;
  const int lx = threadIdx.x & 31;
  int b = box_of(B.tile_off, B.nbox, t0);
  for (int t = t0; t < t1; ++b) {
    const View& v = B.views[b];
    const int base = B.tile_off[b], te = min(t1, B.tile_off[b + 1]);
    const T* __restrict__ fin = static_cast<const T*>(fin_of(v));
    T* __restrict__ fout = static_cast<T*>(fout_of(v));
    const int lg = B.tile_lg, th = 1 << lg;
    const int ntx = (v.nx + 31) >> 5, nty = (v.ny + th - 1) >> lg;
    const int tiles_per_plane = ntx * nty;
    const int nxny = v.nx * v.ny;
    const int rows = (te - t) << lg;   // rows of this block's range in this box
    __syncthreads();
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    auto claim = [&]() {
      int r = 0;
      if (lx == 0) r = atomicAdd(&s_next, 1);
      return __shfl_sync(0xffffffffu, r, 0);
    };
    // row k of the range: tile t + k / th, row k % th of the tile
    auto decode = [&](int k, int& x, int& y, int& z) {
      const int lt = t + (k >> lg) - base;
      z = lt / tiles_per_plane;
      const int r = lt - z * tiles_per_plane;
      const int ty = r / ntx, tx = r - ty * ntx;
      x = tx * 32 + lx;
      y = (ty << lg) + (k & (th - 1));
    };
    TC acc[6] = {0, 0, 0, 0, 0, 0};
    if constexpr (P == 0) {
      for (int k = claim(); k < rows; k = claim()) {
        int x, y, z;
        decode(k, x, y, z);
        const int dzm = z == 0 ? (v.nz - 1) * nxny : -nxny, dzp = z == v.nz - 1 ? (1 - v.nz) * nxny : nxny;
        if (x < v.nx && y < v.ny) {
          // a warp covers one x row, so this branch is warp-uniform
          if (y == 0 || y == v.ny - 1) lb_node<P, true>(v, fin, fout, x, y, z, dzm, dzp, acc);
          else lb_node<P, false>(v, fin, fout, x, y, z, dzm, dzp, acc);
        }
      }
    } else {
      // row pairs (y, y + 1) of a tile (tile heights are even); the tile
      // decode divides by the box's tile counts with one multiply-high each
      FastDiv by_tpp, by_ntx;
      by_tpp.init((uint32_t)tiles_per_plane);
      by_ntx.init((uint32_t)ntx);
      float2 acc2[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) acc2[k] = make_float2(0.0f, 0.0f);
      const int pairs = rows >> 1;
      // tile column x0, first row y and plane z of pair k2
      auto pair_at = [&](int k2, int& x0, int& y, int& z) {
        const int k = 2 * k2;
        const int lt = t + (k >> lg) - base;
        z = (int)by_tpp.div((uint32_t)lt);
        const int r = lt - z * tiles_per_plane;
        const int ty = (int)by_ntx.div((uint32_t)r), tx = r - ty * ntx;
        x0 = tx * 32;
        y = (ty << lg) + (k & (th - 1));
      };
      // both rows off the Lees-Edwards planes (warp-uniform)
      auto interior = [&](int y) { return y >= 1 && y + 1 <= v.ny - 2; };
      auto direct = [&](int x0, int y, int z) {
        const int x = x0 + lx;
        const int dzm = z == 0 ? (v.nz - 1) * nxny : -nxny, dzp = z == v.nz - 1 ? (1 - v.nz) * nxny : nxny;
        if (x >= v.nx || y >= v.ny) return;
        if (!interior(y)) {
          lb_node_single<P>(v, fin, fout, x, y, z, dzm, dzp, acc);
          if (y + 1 < v.ny) lb_node_single<P>(v, fin, fout, x, y + 1, z, dzm, dzp, acc);
        } else if (v.ladd) {
          lb_pair<P, true>(v, fin, fout, x, y, z, dzm, dzp, acc2);
        } else {
          lb_pair<P, false>(v, fin, fout, x, y, z, dzm, dzp, acc2);
        }
      };
      for (int k2 = claim(); k2 < pairs; k2 = claim()) {
        int x0, y, z;
        pair_at(k2, x0, y, z);
        direct(x0, y, z);
      }
      const float vfe = (P == 2) ? v.vf_f * v.inv_scale : v.vf_f;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k] += vfe * (acc2[k].x + acc2[k].y);
    }
    t = te;
    block_sum<TC, 6>(acc, red);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < 6; ++k) atomicAdd(acc_rep(v, blockIdx.x) + k, (double)acc[k]);
  }
}

// ---------------------------------------------------------------------------
// Collide-stream with the source rows staged in shared memory by tensor copies
// (FP32, FP16 and BF16 storage).
//
// A block takes its tiles of 128 (x) by 4 (y) nodes of one z plane in turn.
// For each tile and population p one tensor copy brings the source window of
// p -- x0 - XO .. x0 + 127 + XO (x0 - XO is 16-byte aligned), rows y0 - c_py
// .. y0 - c_py + 3, plane z - c_pz -- into shared memory, all 19 completing
// on the stage's mbarrier.  The copy engine's cost goes with the number of
// box rows, so the windows are wide (288 bytes in 16-bit storage, 544 in
// FP32) and short.  NSTAGE stages are in flight; the last warp to finish a
// tile refills its stage with the tile NSTAGE further on; a 20th copy brings
// the tile's owner words.  Each warp takes one row pair of 32 nodes of a
// tile: interior pairs pull from shared memory (the x-periodic sources of
// the two edge nodes of a row from global memory: staging those as well, by
// 16-byte copies of the rows' other ends, measured slower), Lees-Edwards rows and the last row of an odd L_y take the scalar
// path from global memory.  The per-node arithmetic is that of the row-pair
// path, so the populations equal the direct kernel's bit for bit; the
// viscous sums are reduced per warp instead of per block.  Boxes whose x
// rows are not a multiple of 16 bytes (no tensor map) pull from global
// memory in this kernel too.  Every wait is bounded: a stage that never
// fills raises ERR_TIMEOUT and the block stops after waiting, bounded again,
// for its copies in flight.
// ---------------------------------------------------------------------------
template <int P>
struct TmaShape {
  using T = typename Store<P>::T;
  static constexpr int XO = 16 / (int)sizeof(T);   // window start x0 - XO: 16-byte aligned
  static constexpr int TW = 128;                   // tile width (four 32-node row segments)
  static constexpr int XB = TW + 2 * XO;           // window width (elements)
  static constexpr int TH = 4;                     // tile rows: 8 warps = 4 segments x 2 row pairs
  static constexpr int PLANE = XB * TH;            // elements per population window
  static constexpr int POP_BYTES = 19 * PLANE * (int)sizeof(T);
  static constexpr int OWN_BYTES = TW * TH * 4;                 // the tile's owner words
  static constexpr int STAGE_BYTES = POP_BYTES + OWN_BYTES;
  static constexpr int NSTAGE = sizeof(T) == 4 ? 2 : 4;
  static constexpr int SMEM = NSTAGE * STAGE_BYTES + 8 * NSTAGE + 128;   // + slack to align the base
};
static_assert(TmaShape<1>::SMEM <= 113 * 1024 && TmaShape<2>::SMEM <= 113 * 1024,
              "two staged blocks must fit one SM's shared memory");
static_assert(TmaShape<1>::XB <= 256 && TmaShape<2>::XB <= 256, "tensor-copy box rows hold at most 256 elements");
// every tensor copy lands on a 128-byte boundary of shared memory
static_assert((TmaShape<1>::PLANE * 4) % 128 == 0 && (TmaShape<2>::PLANE * 2) % 128 == 0, "window alignment");
static_assert(TmaShape<1>::POP_BYTES % 128 == 0 && TmaShape<2>::POP_BYTES % 128 == 0, "owner tile alignment");
static_assert(TmaShape<1>::STAGE_BYTES % 128 == 0 && TmaShape<2>::STAGE_BYTES % 128 == 0, "stage alignment");

// Tiles of one box for the staged kernel.
__host__ __device__ inline int tma_tiles(int nx, int ny, int nz) {
  return ((nx + TmaShape<1>::TW - 1) / TmaShape<1>::TW) * ((ny + TmaShape<1>::TH - 1) / TmaShape<1>::TH) * nz;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete; false after about 2^31
// SM cycles (about a second) without it.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  if (mbar_try(a, parity)) return true;
  const long long c0 = clock64();
  while (!mbar_try(a, parity))
    if (clock64() - c0 > (1LL << 31)) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void* map, int x, int y, int z, int q, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(q), "r"(bar)
      : "memory");
}

template <int P> struct Cvt;
template <> struct Cvt<1> { __device__ static float f(float x) { return x; } };
template <> struct Cvt<2> { __device__ static float f(__half x) { return __half2float(x); } };
template <> struct Cvt<3> { __device__ static float f(__nv_bfloat16 x) { return __bfloat162float(x); } };

// Pull of the row pair (x, y), (x, y + 1) from the staged windows st (column
// col = x - x0 of the tile, rows `row` and row + 1); the x-wrap sources of
// the edge nodes (eL: x = 0, eR: x = nx - 1) from global memory, as the
// direct pull takes them.
template <int P, int p>
struct StagedPull {
  using T = typename Store<P>::T;
  __device__ __forceinline__ static void run(const T* st, const T* __restrict__ fin, uint32_t nc, int nx,
                                             uint32_t iA, int col, int row, int dxm, int dxp, int dzm, int dzp,
                                             bool eL, bool eR, bool fA, bool fB, float rest, float2 (&u)[19]) {
    using Sh = TmaShape<P>;
    constexpr int cpx = D3Q19::cx(p), cpy = D3Q19::cy(p), cpz = D3Q19::cz(p);
    const T* s = st + p * Sh::PLANE + row * Sh::XB + (col - cpx + Sh::XO);
    float a = Cvt<P>::f(s[0]), b = Cvt<P>::f(s[Sh::XB]);
    if constexpr (cpx != 0) {
      if (cpx == 1 ? eL : eR) {
        const int off = (cpx == 1 ? dxm : dxp) - cpy * nx + (cpz == 1 ? dzm : (cpz == -1 ? dzp : 0));
        const uint32_t e = (uint32_t)p * nc + iA + (uint32_t)off;
        a = Raw<P>::ld(fin, e);
        b = Raw<P>::ld(fin, e + (uint32_t)nx);
      }
    }
    const float r = (P == 1) ? (float)D3Q19::w(p) * rest : 0.0f;
    u[p].x = fA ? a - r : 0.0f;
    u[p].y = fB ? b - r : 0.0f;
    StagedPull<P, p + 1>::run(st, fin, nc, nx, iA, col, row, dxm, dxp, dzm, dzp, eL, eR, fA, fB, rest, u);
  }
};
template <int P>
struct StagedPull<P, 19> {
  __device__ __forceinline__ static void run(const typename Store<P>::T*, const typename Store<P>::T* __restrict__,
                                             uint32_t, int, uint32_t, int, int, int, int, int, int, bool, bool,
                                             bool, bool, float, float2 (&)[19]) {}
};

// First node (x0, y0) and plane z of staged tile lt of a box.
__device__ __forceinline__ void tma_tile_xyz(const View& v, int lt, int& x0, int& y0, int& z) {
  constexpr int TW = TmaShape<1>::TW, TH = TmaShape<1>::TH;
  const int ntx = (v.nx + TW - 1) / TW, nty = (v.ny + TH - 1) / TH;
  const int tpp = ntx * nty;
  z = lt / tpp;
  const int r = lt - z * tpp;
  const int ty = r / ntx;
  x0 = (r - ty * ntx) * TW;
  y0 = ty * TH;
}

template <int P>
__global__ void __launch_bounds__(256, 2) k_collide_stream_tma(Batch B) {
  using T = typename Store<P>::T;
  using Sh = TmaShape<P>;
  constexpr int NS = Sh::NSTAGE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // tensor copies land on 128-byte boundaries: align the base whatever the
  // static shared memory before it
  unsigned char* const smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t* const full = reinterpret_cast<uint64_t*>(smem + NS * Sh::STAGE_BYTES);
  __shared__ int s_done[NS], s_issued[NS];
  __shared__ int s_abort;
  const int total = B.tile_off[B.nbox];
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  if (t0 >= t1) return;
  const int lx = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(full + s), 1);
      s_done[s] = 0;
      s_issued[s] = 0;
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // tile t into stage s (one thread)
  auto issue = [&](int t, int s) {
    const int b = box_of(B.tile_off, B.nbox, t);
    const View& v = B.views[b];
    const uint32_t bar = smem_u32(full + s);
    ++s_issued[s];
    if (!v.tmap) {
      mbar_arrive(bar);   // this box pulls from global memory
      return;
    }
    int x0, y0, z;
    tma_tile_xyz(v, t - B.tile_off[b], x0, y0, z);
    // maps: [0] fa, [1] fb (the step's source buffer), [2] the owner words
    const char* maps = reinterpret_cast<const char*>(v.tmap);
    const void* map = maps + ((v.proto->t & 1) ? 128 : 0);
    mbar_expect_tx(bar, (uint32_t)Sh::STAGE_BYTES);
    const uint32_t dst = smem_u32(smem + (size_t)s * Sh::STAGE_BYTES);
#pragma unroll
    for (int p = 0; p < 19; ++p)
      tma_load_4d(dst + (uint32_t)(p * Sh::PLANE * sizeof(T)), map, x0 - Sh::XO, y0 - D3Q19::cy(p),
                  wrap1(z - D3Q19::cz(p), v.nz), p, bar);
    tma_load_3d(dst + (uint32_t)Sh::POP_BYTES, maps + 256, x0, y0, z, bar);
  };
  if (threadIdx.x == 0)
    for (int j = 0; j < NS && t0 + j < t1; ++j) issue(t0 + j, j);
  float acc[6] = {0, 0, 0, 0, 0, 0};
  float2 acc2[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) acc2[k] = make_float2(0.0f, 0.0f);
  // this warp's viscous sums into its box's accumulator replica
  auto flush = [&](const View& v) {
    const float vfe = (P == 2) ? v.vf_f * v.inv_scale : v.vf_f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float a = warp_sum_f(acc[k] + vfe * (acc2[k].x + acc2[k].y));
      if (lx == 0) atomicAdd(acc_rep(v, blockIdx.x) + k, (double)a);
      acc[k] = 0.0f;
      acc2[k] = make_float2(0.0f, 0.0f);
    }
  };
  // the current box's constants, reloaded when the tile range enters a box
  int cur = -1;
  const View* vp = B.views;
  const T* fin = nullptr;
  T* fout = nullptr;
  int nx = 0, ny = 0, nz = 0, nxny = 0;
  bool staged = false, ladd = false;
  for (int t = t0, j = 0; t < t1; ++t, ++j) {
    const int s = j % NS;
    const uint32_t par = (uint32_t)(j / NS) & 1u;
    const int b = box_of(B.tile_off, B.nbox, t);
    if (b != cur) {
      if (cur >= 0) flush(*vp);
      cur = b;
      vp = B.views + b;
      fin = static_cast<const T*>(fin_of(*vp));
      fout = static_cast<T*>(fout_of(*vp));
      nx = vp->nx; ny = vp->ny; nz = vp->nz; nxny = nx * ny;
      staged = vp->tmap != nullptr;
      ladd = vp->ladd != 0;
    }
    const View& v = *vp;
    int x0, y0, z;
    tma_tile_xyz(v, t - B.tile_off[b], x0, y0, z);
    // warp w: 32-node segment w & 3, row pair w >> 2 of the tile
    const int col = 32 * (wid & 3) + lx, row = 2 * (wid >> 2);
    const int x = x0 + col, y = y0 + row;
    const bool live = x < nx && y < ny;
    const bool pair = live && y >= 1 && y + 1 <= ny - 2;
    const uint32_t iA = (uint32_t)(x + nx * (y + ny * z));
    // every lane waits (each acquires the copied data); the outcome and the
    // stop decision are taken warp-wide so the warp stays converged
    const bool ok = mbar_wait(smem_u32(full + s), par);
    if (!__all_sync(0xffffffffu, ok) && lx == 0) {
      atomicOr(v.err, ERR_TIMEOUT);
      s_abort = 1;
    }
    if (__any_sync(0xffffffffu, *(volatile int*)&s_abort != 0)) break;
    if (live) {
      const int dzm = z == 0 ? (nz - 1) * nxny : -nxny, dzp = z == nz - 1 ? (1 - nz) * nxny : nxny;
      if (!pair) {
        lb_node_single<P>(v, fin, fout, x, y, z, dzm, dzp, acc);
        if (y + 1 < ny) lb_node_single<P>(v, fin, fout, x, y + 1, z, dzm, dzp, acc);
      } else if (!staged) {
        if (ladd) lb_pair<P, true>(v, fin, fout, x, y, z, dzm, dzp, acc2);
        else lb_pair<P, false>(v, fin, fout, x, y, z, dzm, dzp, acc2);
      } else {
        const unsigned char* st = smem + (size_t)s * Sh::STAGE_BYTES;
        const int* own = reinterpret_cast<const int*>(st + Sh::POP_BYTES) + row * Sh::TW + col;
        const bool fA = own[0] < 0, fB = own[Sh::TW] < 0;
        const int dxm = x == 0 ? nx - 1 : -1, dxp = x == nx - 1 ? 1 - nx : 1;
        const uint32_t nc = (uint32_t)v.ncell;
        float2 u[19];
        StagedPull<P, 0>::run(reinterpret_cast<const T*>(st), fin, nc, nx, iA, col, row, dxm, dxp, dzm, dzp,
                              x == 0, x == nx - 1, fA, fB, v.rho0_f, u);
        if (ladd) pair_collide<P, true>(v, fout, iA, fA, fB, u, acc2);
        else pair_collide<P, false>(v, fout, iA, fA, fB, u, acc2);
      }
    }
    // the stage is read: the last warp to get here refills it
    __syncwarp();
    if (lx == 0) {
      // (the warp's shared-memory reads of the stage are complete: their
      // values went into the stores above)
      if (atomicAdd(&s_done[s], 1) == nwarp - 1) {
        s_done[s] = 0;
        if (t + NS < t1) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(t + NS, s);
        }
      }
    }
  }
  if (cur >= 0) flush(*vp);
  __syncthreads();
  // copies still in flight (only after a timeout): wait for them, bounded,
  // before the block's shared memory is released
  if (threadIdx.x == 0)
    for (int s = 0; s < NS; ++s)
      if (s_issued[s] > 0) mbar_wait(smem_u32(full + s), (uint32_t)(s_issued[s] - 1) & 1u);
}

// Moments (rho, j) of the two Lees-Edwards boundary planes of every box, read
// by the crossing pulls of the next step: plane 0 is y = 0, plane 1 is
// y = ny-1.  The collide-stream writes them for the step after it (the
// plane rows' new populations); this kernel sets them where the populations
// come from elsewhere (creation, set, load).
template <int P>
__global__ void k_plane_moments_b(Batch B) {
  using TC = typename Store<P>::C;
  using T = typename Store<P>::T;
  using S = Store<P>;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B.plane_off[B.nbox]) return;
  const int b = box_of(B.plane_off, B.nbox, g);
  const View& v = B.views[b];
  const T* __restrict__ fin = static_cast<const T*>(fin_of(v));
  const int per = v.nx * v.nz;
  const int l = g - B.plane_off[b];
  const int plane = l / per, r = l - plane * per;
  const int x = r % v.nx, z = r / v.nx;
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
  TC* pm = reinterpret_cast<TC*>(pm_in_of(v)) + 4 * ((long long)plane * per + r);
  pm[0] = rho; pm[1] = jx; pm[2] = jy; pm[3] = jz;
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

// Tiles of the collide-stream grid (upper bound of its block count).
// Collide-stream tiles of one box: 32 x 2^tile_lg nodes, or the staged
// kernel's 128 x 4.
int lb_blocks(int nx, int ny, int nz, int tile_lg, int staged) {
  if (staged) return tma_tiles(nx, ny, nz);
  const int th = 1 << tile_lg;
  return ((nx + 31) / 32) * ((ny + th - 1) / th) * nz;
}

// Dynamic shared memory of the staged kernels, set once per device before
// their first launch or occupancy query (both happen outside graph capture).
static void tma_attrs() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaFuncSetAttribute(k_collide_stream_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaShape<1>::SMEM);
  cudaFuncSetAttribute(k_collide_stream_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaShape<2>::SMEM);
  cudaFuncSetAttribute(k_collide_stream_tma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaShape<3>::SMEM);
  done[dev] = true;
}

// Resident blocks of the collide-stream kernel (direct, or staged: FP32 /
// FP16 / BF16 only) per SM (*per) and the SM count.
void lb_occupancy(int prec, int staged, int* per_sm, int* sms_out) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (staged && prec >= 1) {
    tma_attrs();
    switch (prec) {
      case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_collide_stream_tma<1>, 256, TmaShape<1>::SMEM); break;
      case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_collide_stream_tma<2>, 256, TmaShape<2>::SMEM); break;
      default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_collide_stream_tma<3>, 256, TmaShape<3>::SMEM); break;
    }
  } else {
    switch (prec) {
      case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_collide_stream<0>, 256, 0); break;
      case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_collide_stream<1>, 256, 0); break;
      case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_collide_stream<2>, 256, 0); break;
      default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_collide_stream<3>, 256, 0); break;
    }
  }
  if (e != cudaSuccess || per < 1) per = 1;
  if (sms < 1) sms = 1;
  *per_sm = per;
  *sms_out = sms;
}

// Tensor maps of a box's two population buffers and its owner words for the
// staged kernel, into host memory out[3][128 bytes]: [19][nz][ny][nx]
// elements in windows of TmaShape::XB x TmaShape::TH x 1 x 1 (fa, fb), and
// the [nz][ny][nx] owner words in tiles of TmaShape::TW x TmaShape::TH x 1;
// zero fill outside.  Returns 0 (and the box
// pulls from global memory) for FP64 storage, x rows that are not a
// multiple of 16 bytes, or when the driver offers no encoder.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static std::mutex mu;
  static bool tried = false;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

int lb_tensor_maps(int prec, int nx, int ny, int nz, void* fa, void* fb, void* owner, void* out) {
  if (prec < 1 || prec > 3) return 0;
  const size_t es = prec == 1 ? 4 : 2;
  const int xb = prec == 1 ? TmaShape<1>::XB : TmaShape<2>::XB;
  if ((nx * es) % 16 != 0) return 0;
  if (((uintptr_t)fa | (uintptr_t)fb | (uintptr_t)owner) % 16 != 0) return 0;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return 0;
  const CUtensorMapDataType dt = prec == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : prec == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 19};
  const cuuint64_t strides[3] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es, (cuuint64_t)nx * ny * nz * es};
  const cuuint32_t box[4] = {(cuuint32_t)xb, (cuuint32_t)TmaShape<1>::TH, 1, 1};
  static_assert(TmaShape<1>::TH == TmaShape<2>::TH && TmaShape<1>::TW == TmaShape<2>::TW, "one tile shape");
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUtensorMap* m = static_cast<CUtensorMap*>(out);
  void* bufs[2] = {fa, fb};
  for (int k = 0; k < 2; ++k)
    if (enc(m + k, dt, 4, bufs[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return 0;
  // the owner words [nz][ny][nx] (int32), one tile per copy
  const cuuint64_t odims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t ostr[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t obox[3] = {(cuuint32_t)TmaShape<1>::TW, (cuuint32_t)TmaShape<1>::TH, 1};
  if (enc(m + 2, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, owner, odims, ostr, obox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 0;
  return 1;
}

void launch_plane_moments(int prec, const Batch& B, int total, cudaStream_t s) {
  const int pb = (total + 255) / 256;
  if (pb == 0) return;
  switch (prec) {
    case 0: k_plane_moments_b<0><<<pb, 256, 0, s>>>(B); break;
    case 1: k_plane_moments_b<1><<<pb, 256, 0, s>>>(B); break;
    case 2: k_plane_moments_b<2><<<pb, 256, 0, s>>>(B); break;
    default: k_plane_moments_b<3><<<pb, 256, 0, s>>>(B); break;
  }
}

void launch_collide_stream(int prec, const Batch& B, int grid, int staged, cudaStream_t s) {
  if (staged && prec >= 1) {
    tma_attrs();
    switch (prec) {
      case 1: k_collide_stream_tma<1><<<grid, 256, TmaShape<1>::SMEM, s>>>(B); break;
      case 2: k_collide_stream_tma<2><<<grid, 256, TmaShape<2>::SMEM, s>>>(B); break;
      default: k_collide_stream_tma<3><<<grid, 256, TmaShape<3>::SMEM, s>>>(B); break;
    }
    return;
  }
  switch (prec) {
    case 0: k_collide_stream<0><<<grid, 256, 0, s>>>(B); break;
    case 1: k_collide_stream<1><<<grid, 256, 0, s>>>(B); break;
    case 2: k_collide_stream<2><<<grid, 256, 0, s>>>(B); break;
    default: k_collide_stream<3><<<grid, 256, 0, s>>>(B); break;
  }
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the collide-stream step (particle-free box, FP32).
//
// For callers that cannot allocate device memory or hand the library a
// workspace at all: the two kernels below keep their scratch (the moments of
// the two Lees-Edwards planes and the per-block viscous-stress partials) in
// the file-scope device array susp_noalloc_scratch.  The array is part of the
// library image, so every GPU that loads the library holds it until the
// process exits; all calls share it.
// ---------------------------------------------------------------------------
#include <mutex>

#include "../../include/susp.h"

namespace susp_dev {

constexpr int NOALLOC_MAX_PLANE_NODES = 65536;   // nx * nz
constexpr int NOALLOC_MAX_BLOCKS = 4096;
constexpr size_t NOALLOC_PLANE_BYTES = 2ull * NOALLOC_MAX_PLANE_NODES * 4 * sizeof(float);
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_PLANE_BYTES + 6ull * NOALLOC_MAX_BLOCKS * sizeof(double);

static __device__ __align__(256) unsigned char susp_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

struct NoAllocLE {
  int di;
  float w_lo, w_hi, ule;   // interpolation weights on c1 (y = 0 / y = ny-1 receivers), U_LE
};

// Fluid-only pull across a Lees-Edwards plane: linear interpolation between
// the two straddling nodes plus the Galilean correction with their moments.
template <int p>
__device__ __forceinline__ float noalloc_le_pull(const View& v, const float* __restrict__ fin,
                                                 const float* __restrict__ pm_all, NoAllocLE le,
                                                 int x, int z) {
  const int nx = v.nx, ny = v.ny;
  const long long nc = v.ncell;
  constexpr int cpx = D3Q19::cx(p), cpy = D3Q19::cy(p), cpz = D3Q19::cz(p);
  const bool below = (cpy == 1);
  const int sx = x - cpx, sz = wrapi(z - cpz, v.nz);
  const int ys = below ? ny - 1 : 0;
  const int c0x = below ? wrapi(sx + le.di, nx) : wrapi(sx - le.di - 1, nx);
  const int c1x = c0x + 1 == nx ? 0 : c0x + 1;
  const float w1 = below ? le.w_lo : le.w_hi;
  const long long i0 = c0x + (long long)nx * (ys + (long long)ny * sz);
  const long long i1 = c1x + (long long)nx * (ys + (long long)ny * sz);
  const float* pm = pm_all + (below ? 4LL * v.nz * nx : 0);
  const long long k0 = 4LL * (c0x + (long long)nx * sz), k1 = 4LL * (c1x + (long long)nx * sz);
  const float a = 1.0f - w1;
  float val = a * __ldg(fin + (long long)p * nc + i0) + w1 * __ldg(fin + (long long)p * nc + i1);
  const float rho = a * pm[k0] + w1 * pm[k1];
  const float jx = a * pm[k0 + 1] + w1 * pm[k1 + 1];
  const float jy = a * pm[k0 + 2] + w1 * pm[k1 + 2];
  const float jz = a * pm[k0 + 3] + w1 * pm[k1 + 3];
  const float sgn = below ? -1.0f : 1.0f;
  const float inv = 1.0f / rho;
  val += feq<float>(p, rho, jx + sgn * rho * le.ule, jy, jz, inv) - feq<float>(p, rho, jx, jy, jz, inv);
  return val;
}

template <int p>
struct NoAllocPull {
  __device__ __forceinline__ static void run(const View& v, const float* __restrict__ fin,
                                             const float* __restrict__ pm, NoAllocLE le, int x, int y,
                                             int z, int xm, int xp, int zm, int zp, float (&n)[19]) {
    constexpr int cpx = D3Q19::cx(p), cpy = D3Q19::cy(p), cpz = D3Q19::cz(p);
    const int sy = y - cpy;
    if (cpy != 0 && (sy < 0 || sy >= v.ny)) {
      n[p] = noalloc_le_pull<p>(v, fin, pm, le, x, z);
    } else {
      const int sx = cpx == 1 ? xm : (cpx == -1 ? xp : x);
      const int sz = cpz == 1 ? zm : (cpz == -1 ? zp : z);
      n[p] = __ldg(fin + (long long)p * v.ncell + sx + (long long)v.nx * (sy + (long long)v.ny * sz));
    }
    NoAllocPull<p + 1>::run(v, fin, pm, le, x, y, z, xm, xp, zm, zp, n);
  }
};
template <>
struct NoAllocPull<19> {
  __device__ __forceinline__ static void run(const View&, const float* __restrict__, const float* __restrict__,
                                             NoAllocLE, int, int, int, int, int, int, int, float (&)[19]) {}
};

__global__ void __launch_bounds__(256) k_fluid_step_noalloc(View v, const float* __restrict__ fin,
                                                            float* __restrict__ fout, NoAllocLE le,
                                                            double* __restrict__ partials) {
  __shared__ float red[32 * 6];
  float acc[6] = {0, 0, 0, 0, 0, 0};
  const float* pm = reinterpret_cast<const float*>(v.plane_mom);
  const int ntx = (v.nx + 31) >> 5, nty = (v.ny + 7) >> 3;
  const int tiles_per_plane = ntx * nty;
  const long long ntiles = (long long)tiles_per_plane * v.nz;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const float omega = v.omega_f, vf = v.vf_f;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int z = (int)(t / tiles_per_plane);
    const int r = (int)(t - (long long)z * tiles_per_plane);
    const int ty = r / ntx, tx = r - ty * ntx;
    const int x = tx * 32 + lx, y = ty * 8 + ly;
    if (x >= v.nx || y >= v.ny) continue;
    const long long idx = x + (long long)v.nx * (y + (long long)v.ny * z);
    const int xm = x == 0 ? v.nx - 1 : x - 1, xp = x == v.nx - 1 ? 0 : x + 1;
    const int zm = z == 0 ? v.nz - 1 : z - 1, zp = z == v.nz - 1 ? 0 : z + 1;
    float n[19];
    n[0] = __ldg(fin + idx);
    NoAllocPull<1>::run(v, fin, pm, le, x, y, z, xm, xp, zm, zp, n);
    // second moments from the deviations n - C^q (rho0 = 1; exact
    // differences), so that Pi - rho I / 3 cancels no values of size 1/3
    float rho = 0, rdev = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      const float cxq = (float)D3Q19::cx(q), cyq = (float)D3Q19::cy(q), czq = (float)D3Q19::cz(q);
      const float d = n[q] - (float)D3Q19::w(q);
      rho += n[q];
      rdev += d;
      jx += n[q] * cxq; jy += n[q] * cyq; jz += n[q] * czq;
      pxx += d * cxq * cxq; pyy += d * cyq * cyq; pzz += d * czq * czq;
      pxy += d * cxq * cyq; pxz += d * cxq * czq; pyz += d * cyq * czq;
    }
    const float inv = 1.0f / rho;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      const float fe = feq<float>(q, rho, jx, jy, jz, inv);
      fout[(long long)q * v.ncell + idx] = n[q] - omega * (n[q] - fe);
    }
    const float third = rdev / 3.0f;
    acc[0] += vf * (pxx - jx * jx * inv - third);
    acc[1] += vf * (pyy - jy * jy * inv - third);
    acc[2] += vf * (pzz - jz * jz * inv - third);
    acc[3] += vf * (pxy - jx * jy * inv);
    acc[4] += vf * (pxz - jx * jz * inv);
    acc[5] += vf * (pyz - jy * jz * inv);
  }
  block_sum<float, 6>(acc, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) partials[6LL * blockIdx.x + k] = (double)acc[k];
}

// Sums the per-block partials in block order and writes the 3 x 3 viscous
// stress of the step (divided by the box volume); overwrites out.
__global__ void k_fluid_visc_noalloc(const double* __restrict__ partials, int nblk, double inv_volume,
                                     double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nblk; ++b)
    for (int k = 0; k < 6; ++k) s[k] += partials[6LL * b + k];
  const double full[9] = {s[0], s[3], s[4], s[3], s[1], s[5], s[4], s[5], s[2]};
  for (int k = 0; k < 9; ++k) out[k] = full[k] * inv_volume;
}

}  // namespace susp_dev

namespace {
// The scratch array's device address belongs to one CUDA context: a device
// reset, or another context made current on this device, loads the library's
// module again at another address.  The address is therefore cached per
// device together with the unique ID of the context it was looked up in
// (cuCtxGetId, reached through the runtime's driver entry points so that the
// library does not link libcuda), and looked up again when the current
// context's ID differs.
std::mutex g_noalloc_mu;
struct NoAllocAddr {
  unsigned long long ctx_id;
  void* ptr;
};
NoAllocAddr g_noalloc_addr[256];
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_ctx_fns_tried = false;

// ID of the context current on this thread; 0 if there is none yet or the
// driver entry points are unavailable (the caller then looks the address up
// on every call).  Called with g_noalloc_mu held.
unsigned long long current_ctx_id() {
  if (!g_ctx_fns_tried) {
    g_ctx_fns_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(fn);
  }
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
  if (g_ctx_get_id(ctx, &id) != 0) return 0;
  return id;
}
}  // namespace

void susp_set_last_error(const char* msg);

extern "C" susp_status susp_fluid_step_noalloc(int nx, int ny, int nz, double tau, double delta, double u_le,
                                               const float* f_in, float* f_out, double* visc_out,
                                               void* cuda_stream) {
  using namespace susp_dev;
  if (nx < 4 || ny < 4 || nz < 4 || !(tau > 0.5) || !f_in || !f_out || !visc_out) {
    susp_set_last_error("susp_fluid_step_noalloc: bad argument");
    return SUSP_EINVAL;
  }
  if ((long long)nx * nz > NOALLOC_MAX_PLANE_NODES || (long long)nx * ny * nz >= (1LL << 31)) {
    susp_set_last_error("susp_fluid_step_noalloc: nx * nz exceeds 65536 (the size of its static scratch)");
    return SUSP_EINVAL;
  }
  {
    // the step reads f_in while it writes f_out: the two ranges must be disjoint
    const unsigned long long bytes = 19ull * (unsigned long long)nx * ny * nz * sizeof(float);
    const unsigned long long a0 = (unsigned long long)(uintptr_t)f_in, b0 = (unsigned long long)(uintptr_t)f_out;
    if (a0 < b0 + bytes && b0 < a0 + bytes) {
      susp_set_last_error("susp_fluid_step_noalloc: f_in and f_out overlap");
      return SUSP_EINVAL;
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    susp_set_last_error("susp_fluid_step_noalloc: no current CUDA device");
    return SUSP_ECUDA;
  }
  void* scratch = nullptr;
  {
    // first call in this device's current context: look up the device
    // address of the static array
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocAddr& A = g_noalloc_addr[dev];
    unsigned long long id = current_ctx_id();
    if (!A.ptr || id == 0 || id != A.ctx_id) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, susp_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        A.ptr = nullptr;
        A.ctx_id = 0;
        susp_set_last_error("susp_fluid_step_noalloc: cudaGetSymbolAddress failed");
        return SUSP_ECUDA;
      }
      if (id == 0) id = current_ctx_id();   // the look-up made the primary context current
      A.ptr = ptr;
      A.ctx_id = id;
    }
    scratch = A.ptr;
  }
  View v;
  memset(&v, 0, sizeof v);
  v.nx = nx; v.ny = ny; v.nz = nz;
  v.ncell = (long long)nx * ny * nz;
  v.tau = tau; v.rho0 = 1.0; v.rho0_f = 1.0f;
  v.omega_d = 1.0 / tau; v.vf_d = -(1.0 - 0.5 / tau);
  v.omega_f = (float)v.omega_d; v.vf_f = (float)v.vf_d;
  v.scale = 1.0f; v.inv_scale = 1.0f;
  v.plane_mom = scratch;
  double* partials = reinterpret_cast<double*>(static_cast<char*>(scratch) + NOALLOC_PLANE_BYTES);
  // offset split exactly as the library's protocol state does it
  const double dm = delta - nx * floor(delta / nx);
  NoAllocLE le;
  le.di = (int)floor(dm);
  const double w = dm - le.di;
  le.w_lo = (float)w;
  le.w_hi = (float)(1.0 - w);
  le.ule = (float)u_le;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = ((nx + 31) / 32) * ((ny + 7) / 8) * nz;
  int nblk = (sms > 0 ? sms : 1) * 4;
  if (nblk > tiles) nblk = tiles;
  if (nblk > NOALLOC_MAX_BLOCKS) nblk = NOALLOC_MAX_BLOCKS;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long per = 2LL * nx * nz;
  k_plane_moments<1><<<(int)((per + 255) / 256), 256, 0, s>>>(v, f_in);
  k_fluid_step_noalloc<<<nblk, 256, 0, s>>>(v, f_in, f_out, le, partials);
  k_fluid_visc_noalloc<<<1, 32, 0, s>>>(partials, nblk, 1.0 / ((double)nx * ny * nz), visc_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    susp_set_last_error(cudaGetErrorString(e));
    return SUSP_ECUDA;
  }
  return SUSP_OK;
}
