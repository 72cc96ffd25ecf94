// couple.cu — fluid-particle coupling on the node map (Appendix A).
//
// Nodes closer than the mapped radius a_map = 0.95 a to a particle centre
// (any Lees-Edwards image) are solid and owned by that particle.  After the
// particles move:
//   k_uncover: solid nodes that left the mapped sphere become fluid with
//              n = n^eq(rho0, rho0 u_b); the particle loses that momentum
//              (and its moment about the centre);
//   k_cover:   fluid nodes that entered become solid; their momentum
//              sum_q n_q c_q goes to the particle;
//   k_links:   for every solid node s of the particle and direction p, the
//              fluid node r that pulls population p from s (r = s + c_p, or
//              across a Lees-Edwards plane the node whose nearest source is
//              s) forms a boundary link.  It contributes the momentum
//              exchange f = [2 n*_q(r) - 6 C^q rho0 (u_b . c_q)] c_q, q = -p
//              (Eq. 6), to F^h (Eq. 9), (r_b - R) x f to T^h (Eq. 10) and
//              (r_b - R)_a f_b to the particle stresslet (sigma^h); and for a
//              link that does not cross a Lees-Edwards plane it stores the
//              bounce-back value of Eq. 7, n*_q(r) - 6 C^q rho0 (u_b . c_q),
//              in the population slot p of the solid node s.  That slot is
//              exactly what the next collide-stream pulls for (r, p) (r - c_p
//              = s), and no other receiver pulls it, so the lattice kernel
//              streams plainly over solid sources.  A node of another
//              particle j in place of r (mapped spheres closer than one
//              spacing) counts as fluid in equilibrium moving with the mean
//              ubar of the two surfaces' velocities at r_b, against a wall
//              moving with ubar: f = C^q rho0 (2 + 9 (ubar.c_q)^2 -
//              3 ubar^2) c_q.  The pressure on each particle then balances at
//              rest and in a flow moving with both, and the reverse link of j
//              cancels it exactly.
// One block per particle scans the cells of the particle's bounding boxes
// (one per Lees-Edwards image that reaches into the box).  Per-particle sums
// use a fixed-order block reduction, so they are deterministic.
#include <type_traits>

#include "susp_dev.cuh"

namespace susp_dev {

// Bounding box of one Lees-Edwards image of a particle: first node, extents,
// node count, and the image centre (x brought into [0, nx)).
template <typename TC>
struct ImgBox {
  int x0, y0, z0, ex, ey, ez, cnt;
  TC cx, cy, cz;
};

template <typename TC>
__device__ inline int particle_boxes(const View& v, TC Rx, TC Ry, TC Rz, TC delta, TC reach,
                                     ImgBox<TC> (&b)[3]) {
  int total = 0;
#pragma unroll
  for (int k = -1; k <= 1; ++k) {
    ImgBox<TC>& B = b[k + 1];
    // image centre, x brought back into [0, nx): Rx + k delta can lie up to one
    // period outside (0 <= delta < nx), and the cell visit wraps x only once
    TC cx = Rx + (TC)k * delta;
    cx -= (TC)v.nx * floor(cx * sel<TC>(v.inv_nx_d, v.inv_nx_f));
    const TC cy = Ry + (TC)k * (TC)v.ny, cz = Rz;
    int y0 = (int)ceil(cy - reach), y1 = (int)floor(cy + reach);
    if (y0 < 0) y0 = 0;
    if (y1 > v.ny - 1) y1 = v.ny - 1;
    const int x0 = (int)ceil(cx - reach), x1 = (int)floor(cx + reach);
    const int z0 = (int)ceil(cz - reach), z1 = (int)floor(cz + reach);
    B.x0 = x0; B.y0 = y0; B.z0 = z0;
    B.ex = x1 - x0 + 1; B.ey = y1 - y0 + 1; B.ez = z1 - z0 + 1;
    B.cx = cx; B.cy = cy; B.cz = cz;
    B.cnt = (y0 > y1) ? 0 : B.ex * B.ey * B.ez;
    total += B.cnt;
  }
  return total;
}

// Whether node (xu, y, zu) (unwrapped coordinates of image k's box) lies
// inside particle i's mapped sphere, decided from the FP64 centre and offset
// as the oracle decides it.  Out of line: it runs only for the rare nodes
// whose FP32 distance lies within rounding of the surface.
__device__ __noinline__ bool inside_fp64(const View& v, int i, int k, int xu, int y, int zu) {
  const double cx = v.R[3 * i] + (double)k * v.proto->delta;
  const double cy = v.R[3 * i + 1] + (double)k * (double)v.ny, cz = v.R[3 * i + 2];
  double ex = (double)xu - cx, ey = (double)y - cy, ez = (double)zu - cz;
  // the FP32 box may have wrapped the centre by one period where FP64 does
  // not (a centre within rounding of x = 0 or L_x): take the nearest image
  ex -= (double)v.nx * floor(ex * v.inv_nx_d + 0.5);
  ez -= (double)v.nz * floor(ez * v.inv_nz_d + 0.5);
  return ex * ex + (ey * ey + ez * ez) < v.amap[i] * v.amap[i];
}

// Visit the cells of a particle's image boxes: half-warps take (y, z) rows and
// their 16 lanes run along x (coalesced).  Box corners lie less than one period
// outside the lattice (reach < L / 2, centres in [0, L)), so one wrap suffices.
// fn(x, y, z, c, dx, dy, dz, k) gets the cell index and the displacement from
// the particle's image k: every node of an image's box lies within reach of
// that image's centre (reach < L / 2, the boxes of different images do not
// overlap), so that image is the node's minimum image and the displacement is
// the unwrapped coordinate minus the image centre.
// Rows (y, z) whose distance from the image's x axis is row_r or more (plus
// the FP64 window below) hold no node closer than row_r and are skipped.  fn
// also gets d2 = dx^2 + (dy^2 + dz^2), summed in that order so that the row
// test and every node test agree.  ip and am are the particle's index and
// mapped radius (for the FP64 decision near the surface).
template <typename TC, typename F>
__device__ __forceinline__ void for_box_cells(const View& v, const ImgBox<TC> (&b)[3], TC Rx, TC Ry, TC Rz,
                                              TC delta, TC row_r, F&& fn, int ip, TC am) {
  // FP32 centres carry up to half an ulp of the box size (~4e-6 at L = 96),
  // which moves d2 by up to ~3.5 a_map ulp(L); nodes whose d2 lies within
  // twice that of a_map^2 are decided in FP64, so every kernel testing
  // d2 < am * am (claim, uncover, cover, links) takes the oracle's decision
  const TC win = (TC)(4.0 * 1.2e-7) * am * (TC)max(v.nx, max(v.ny, v.nz)) + (TC)1e-5;
  const TC row_r2 = row_r * row_r + (sizeof(TC) == 4 ? (TC)2 * win : (TC)0);
  const TC am2 = am * am;
  const int lane = threadIdx.x & 15, half = threadIdx.x >> 4, nhalf = blockDim.x >> 4;
#pragma unroll
  for (int kb = 0; kb < 3; ++kb) {
    const ImgBox<TC> B = b[kb];
    if (B.cnt == 0) continue;
    const int rows = B.ey * B.ez;
    for (int row = half; row < rows; row += nhalf) {
      const int lz = row / B.ey, ly = row - lz * B.ey;
      const int y = B.y0 + ly, zu = B.z0 + lz, z = wrap1(zu, v.nz);
      const TC dy = (TC)y - B.cy, dz = (TC)zu - B.cz;
      const TC rho2 = dy * dy + dz * dz;
      if (!(rho2 < row_r2)) continue;
      for (int lx = lane; lx < B.ex; lx += 16) {
        const int xu = B.x0 + lx, x = wrap1(xu, v.nx);
        const TC dx = (TC)xu - B.cx;
        const int k = kb - 1;
        const long long c = x + (long long)v.nx * (y + (long long)v.ny * z);
        TC d2 = dx * dx + rho2;
        if constexpr (sizeof(TC) == 4) {
          if (fabsf(d2 - am2) < win)
            d2 = inside_fp64(v, ip, k, xu, y, zu) ? fminf(d2, nextafterf(am2, 0.0f)) : fmaxf(d2, am2);
        }
        fn(x, y, z, c, dx, dy, dz, k, d2);
      }
    }
  }
}

template <typename TC>
__device__ inline TC pdelta(const Proto* pr) { return sel<TC>(pr->delta, pr->delta_f); }
template <typename TC>
__device__ inline TC pule(const Proto* pr) { return sel<TC>(pr->ule, pr->ule_f); }

// Initial claim of the solid nodes (creation).
template <int P>
__global__ void k_claim(Batch B) {
  using TC = typename Store<P>::C;
  const int g = blockIdx.x;
  const int bx = box_of(B.part_off, B.nbox, g);
  const View& v = B.views[bx];
  const int i = g - B.part_off[bx];
  const TC* pp = reinterpret_cast<const TC*>(v.plb) + 12 * i;
  const TC Rx = pp[0], Ry = pp[1], Rz = pp[2];
  const TC am = sel<TC>(v.amap[i], (float)v.amap[i]);
  const TC delta = pdelta<TC>(v.proto);
  ImgBox<TC> b[3];
  particle_boxes<TC>(v, Rx, Ry, Rz, delta, am + (TC)1, b);
  for_box_cells<TC>(v, b, Rx, Ry, Rz, delta, am, [&](int, int, int, long long c, TC, TC, TC, int, TC d2) {
    if (d2 < am * am) {
      const int old = atomicCAS(v.owner + c, -1, i);
      if (old != -1 && old != i) atomicOr(v.err, ERR_OVERLAP);
    }
  }, i, am);
}

// Band nodes of one particle collected by the scan of its bounding boxes, so
// that their owner words are then loaded in one round by all threads instead
// of one dependent load per scan step.  A node that finds the list full is
// handled where the scan met it.
constexpr int BAND_CAP = 1024;
template <typename TC>
struct BandList {
  uint32_t c[BAND_CAP];   // node index (19 ncell < 2^32)
  TC d[BAND_CAP][3];      // displacement from the particle's image centre
  signed char k[BAND_CAP];
  int n;
};

template <typename TC>
__device__ __forceinline__ bool band_push(BandList<TC>& L, long long c, TC dx, TC dy, TC dz, int k) {
  const int slot = atomicAdd(&L.n, 1);
  if (slot >= BAND_CAP) return false;
  L.c[slot] = (uint32_t)c;
  L.d[slot][0] = dx; L.d[slot][1] = dy; L.d[slot][2] = dz;
  L.k[slot] = (signed char)k;
  return true;
}

// WIDE: at most 64 registers (a few spilled) so that more blocks share an
// SM, for launches of many waves (large batches).
template <int P, bool WIDE>
__global__ void __launch_bounds__(256, P == 0 ? 2 : (WIDE ? 4 : 3)) k_uncover(Batch B) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  __shared__ TC red[32 * 6];
  __shared__ BandList<TC> L;
  const int g = blockIdx.x;
  const int bx = box_of(B.part_off, B.nbox, g);
  const View& v = B.views[bx];
  const int i = g - B.part_off[bx];
  typename Store<P>::T* __restrict__ f = static_cast<typename Store<P>::T*>(fin_of(v));
  const TC* pp = reinterpret_cast<const TC*>(v.plb) + 12 * i;
  const TC Rx = pp[0], Ry = pp[1], Rz = pp[2];
  const TC am = sel<TC>(v.amap[i], (float)v.amap[i]);
  const TC delta = pdelta<TC>(v.proto), ule = pule<TC>(v.proto);
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
  if (threadIdx.x == 0) L.n = 0;
  __syncthreads();
  ImgBox<TC> b[3];
  particle_boxes<TC>(v, Rx, Ry, Rz, delta, am + (TC)0.6, b);   // the band's outer radius
  TC acc[6] = {0, 0, 0, 0, 0, 0};
  // solid node of this particle that left the mapped sphere: fluid at rho0
  // and the boundary velocity; the particle loses that momentum
  auto release = [&](long long c, TC dx, TC dy, TC dz, int k) {
    if (v.owner[c] != i) return;
    const TC ubx = pp[3] + (pp[7] * dz - pp[8] * dy) + (TC)k * ule;
    const TC uby = pp[4] + (pp[8] * dx - pp[6] * dz);
    const TC ubz = pp[5] + (pp[6] * dy - pp[7] * dx);
    const TC jx = rho0 * ubx, jy = rho0 * uby, jz = rho0 * ubz;
    const TC inv = (TC)1 / rho0;
#pragma unroll
    for (int q = 0; q < 19; ++q)
      f[(long long)q * v.ncell + c] =
          S::enc(feq<TC>(q, rho0, jx, jy, jz, inv), (TC)D3Q19::w(q) * rho0, (TC)v.scale);
    v.owner[c] = -1;
    {
      // a node of a Lees-Edwards plane: the moments its crossing pulls read
      const long long nxy = (long long)v.nx * v.ny;
      const int y = (int)((c % nxy) / v.nx);
      if (y == 0 || y == v.ny - 1) {
        const long long x = c % v.nx, z = c / nxy;
        TC* pm = reinterpret_cast<TC*>(pm_in_of(v)) + 4 * ((y == 0 ? 0 : (long long)v.nz * v.nx) + x + v.nx * z);
        pm[0] = rho0; pm[1] = jx; pm[2] = jy; pm[3] = jz;
      }
    }
    acc[0] -= jx; acc[1] -= jy; acc[2] -= jz;
    acc[3] -= dy * jz - dz * jy; acc[4] -= dz * jx - dx * jz; acc[5] -= dx * jy - dy * jx;
  };
  for_box_cells<TC>(v, b, Rx, Ry, Rz, delta, am + (TC)0.6,
                    [&](int, int, int, long long c, TC dx, TC dy, TC dz, int k, TC d2) {
    // only nodes outside the mapped sphere can leave it, and only those that
    // were inside before the move: closer than a_map + 0.5 (a particle moves
    // less than 0.5 per step; 0.6 leaves a margin)
    if (d2 < am * am || !(d2 < (am + (TC)0.6) * (am + (TC)0.6))) return;
    if (!band_push(L, c, dx, dy, dz, k)) release(c, dx, dy, dz, k);
  }, i, am);
  __syncthreads();
  const int n = min(L.n, BAND_CAP);
  for (int e = threadIdx.x; e < n; e += blockDim.x)
    release((long long)L.c[e], L.d[e][0], L.d[e][1], L.d[e][2], (int)L.k[e]);
  block_sum<TC, 6>(acc, red);
  if (threadIdx.x == 0) {
    for (int a = 0; a < 3; ++a) {
      v.Fcov[3 * i + a] = (double)acc[a];
      v.Tcov[3 * i + a] = (double)acc[3 + a];
    }
  }
}

template <int P>
__global__ void __launch_bounds__(256, P == 0 ? 2 : 4) k_cover(Batch B) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  __shared__ TC red[32 * 6];
  __shared__ BandList<TC> L;
  const int g = blockIdx.x;
  const int bx = box_of(B.part_off, B.nbox, g);
  const View& v = B.views[bx];
  const int i = g - B.part_off[bx];
  const typename Store<P>::T* __restrict__ f = static_cast<const typename Store<P>::T*>(fin_of(v));
  const TC* pp = reinterpret_cast<const TC*>(v.plb) + 12 * i;
  const TC Rx = pp[0], Ry = pp[1], Rz = pp[2];
  const TC am = sel<TC>(v.amap[i], (float)v.amap[i]);
  const TC delta = pdelta<TC>(v.proto);
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
  if (threadIdx.x == 0) L.n = 0;
  __syncthreads();
  ImgBox<TC> b[3];
  particle_boxes<TC>(v, Rx, Ry, Rz, delta, am, b);   // nodes inside the mapped sphere only
  TC acc[6] = {0, 0, 0, 0, 0, 0};
  const TC inner = am > (TC)0.6 ? am - (TC)0.6 : (TC)0;
  // fluid node that entered the mapped sphere: solid, its momentum goes to
  // the particle (a node held by another particle is an overlap)
  auto claim = [&](long long c, TC dx, TC dy, TC dz) {
    const int own = v.owner[c];
    if (own == i) return;
    const int old = own == -1 ? atomicCAS(v.owner + c, -1, i) : own;
    if (old != -1) { atomicOr(v.err, ERR_OVERLAP); return; }
    TC jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      const TC fq = S::load(f, (long long)q * v.ncell + c, (TC)D3Q19::w(q) * rho0, (TC)v.inv_scale);
      jx += fq * (TC)D3Q19::cx(q); jy += fq * (TC)D3Q19::cy(q); jz += fq * (TC)D3Q19::cz(q);
    }
    acc[0] += jx; acc[1] += jy; acc[2] += jz;
    acc[3] += dy * jz - dz * jy; acc[4] += dz * jx - dx * jz; acc[5] += dx * jy - dy * jx;
  };
  for_box_cells<TC>(v, b, Rx, Ry, Rz, delta, am, [&](int, int, int, long long c, TC dx, TC dy, TC dz, int k, TC d2) {
    // nodes deeper than a_map - 0.6 were inside before the move (speed < 0.5)
    if (!(d2 < am * am) || d2 < inner * inner) return;
    if (!band_push(L, c, dx, dy, dz, k)) claim(c, dx, dy, dz);
  }, i, am);
  __syncthreads();
  const int n = min(L.n, BAND_CAP);
  for (int e = threadIdx.x; e < n; e += blockDim.x) claim((long long)L.c[e], L.d[e][0], L.d[e][1], L.d[e][2]);
  block_sum<TC, 6>(acc, red);
  if (threadIdx.x == 0) {
    for (int a = 0; a < 3; ++a) {
      v.Fcov[3 * i + a] += (double)acc[a];
      v.Tcov[3 * i + a] += (double)acc[3 + a];
    }
  }
}

// Node that pulls population p (components cp) from solid node (x, y, z);
// returns its index (< 2^27 nodes per box).  crossing = the pull passes a
// Lees-Edwards plane.
__device__ __forceinline__ uint32_t link_target_nr(const View& v, const Proto* pr, int x, int y, int z,
                                                   int4 cp, int& rx, int& ry, int& rz, bool& crossing) {
  const int cpx = cp.x, cpy = cp.y, cpz = cp.z;
  ry = y + cpy;
  rz = z + cpz;
  if (rz < 0) rz += v.nz;
  else if (rz >= v.nz) rz -= v.nz;
  crossing = (ry < 0) || (ry >= v.ny);
  int xx;
  if (!crossing) {
    xx = x + cpx;
  } else if (ry >= v.ny) {
    // receiver at y = 0 pulls from below: nearest source x_r - c_px + di + near_lo
    ry = 0;
    xx = x + cpx - pr->di - pr->near_lo;
  } else {
    // receiver at y = ny-1 pulls from above: nearest source x_r - c_px - di - 1 + near_hi
    ry = v.ny - 1;
    xx = x + cpx + pr->di + 1 - pr->near_hi;
  }
  rx = crossing ? wrapi(xx, v.nx) : wrap1(xx, v.nx);
  return (uint32_t)(rx + v.nx * (ry + v.ny * rz));
}

// Momentum exchange of a link from node (rx, ry, rz) of particle j into the
// solid of a particle whose boundary velocity there is ub (direction q into
// that solid): the node stands for fluid in equilibrium moving with the mean
// ubar of the two surfaces' velocities at r_b = r + c_q / 2, against a wall
// moving with ubar, 2 n^eq_q(rho0, rho0 ubar) - 6 C^q rho0 ubar.c_q =
// C^q rho0 (2 + 9 (ubar.c_q)^2 - 3 ubar^2).  Such links are rare (mapped
// spheres closer than one spacing); kept out of line so that their registers
// do not weigh on the link loop.
template <typename TC>
__device__ __noinline__ TC touching_link(const View& v, int j, int rx, int ry, int rz, int q, TC ubx, TC uby,
                                         TC ubz, TC delta, TC ule, TC rho0) {
  const TC cqx = (TC)D3Q19::cx(q), cqy = (TC)D3Q19::cy(q), cqz = (TC)D3Q19::cz(q);
  const TC* pj = reinterpret_cast<const TC*>(v.plb) + 12 * j;
  TC ex = (TC)rx + (TC)0.5 * cqx - pj[0], ey = (TC)ry + (TC)0.5 * cqy - pj[1], ez = (TC)rz + (TC)0.5 * cqz - pj[2];
  const int kj = le_image_v(v, ex, ey, ez, delta);
  const TC mx = (TC)0.5 * (ubx + pj[3] + (pj[7] * ez - pj[8] * ey) + (TC)kj * ule);
  const TC my = (TC)0.5 * (uby + pj[4] + (pj[8] * ex - pj[6] * ez));
  const TC mz = (TC)0.5 * (ubz + pj[5] + (pj[6] * ey - pj[7] * ex));
  const TC cm = mx * cqx + my * cqy + mz * cqz;
  return wq<TC>(q) * rho0 * ((TC)2 + (TC)9 * cm * cm - (TC)3 * (mx * mx + my * my + mz * mz));
}

// Links of one particle in two passes: the block first collects its solid
// nodes near the mapped surface into shared memory, then its threads take
// (node, direction) work items, so every lane does the same work.
constexpr int LINK_NODES_MAX = 2048;
constexpr int LINK_CHUNK = 4608;     // items of one round: up to 18 per node, one node per thread of 256

// WIDE: four resident blocks per SM (64 registers, a few spilled) instead of
// three, for launches of many waves (large batches), where the extra warps
// hide more latency than the spills cost; with one or two waves the
// three-block form is faster.
template <int P, bool WIDE>
__global__ void __launch_bounds__(256, P == 0 ? 2 : (WIDE ? 4 : 3)) k_links(Batch B) {
  using TC = typename Store<P>::C;
  using S = Store<P>;
  __shared__ TC red[32 * 15];
  __shared__ int s_nodes, s_items_n;
  __shared__ uint32_t s_node[LINK_NODES_MAX];   // packed (x, y, z) of solid surface nodes
  __shared__ uint32_t s_mask[LINK_NODES_MAX];   // their candidate link directions (bits 1-18)
  __shared__ uint32_t s_items[LINK_CHUNK];      // (node << 5 | direction) items of one round
  __shared__ int4 s_cp[19];                     // c_p of each direction p
  __shared__ typename std::conditional<sizeof(TC) == 8, double4, float4>::type s_cq[19];   // c_q, C^q of q = -p
  const int g = blockIdx.x;
  const int bx = box_of(B.part_off, B.nbox, g);
  const View& v = B.views[bx];
  const int i = g - B.part_off[bx];
  typename Store<P>::T* __restrict__ f = static_cast<typename Store<P>::T*>(fin_of(v));
  if (threadIdx.x == 0) { s_nodes = 0; s_items_n = 0; }
  if (threadIdx.x < 19) {
    // direction tables: the items index them with a runtime direction
    const int p = threadIdx.x;
    s_cp[p] = make_int4(D3Q19::cx(p), D3Q19::cy(p), D3Q19::cz(p), 0);
    s_cq[p].x = (TC)-D3Q19::cx(p); s_cq[p].y = (TC)-D3Q19::cy(p); s_cq[p].z = (TC)-D3Q19::cz(p);
    s_cq[p].w = (TC)D3Q19::w(p);
  }
  __syncthreads();
  const TC* pp = reinterpret_cast<const TC*>(v.plb) + 12 * i;
  const TC Rx = pp[0], Ry = pp[1], Rz = pp[2];
  const TC am = sel<TC>(v.amap[i], (float)v.amap[i]);
  const Proto* pr = v.proto;
  const TC delta = pdelta<TC>(pr), ule = pule<TC>(pr);
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
  ImgBox<TC> b[3];
  particle_boxes<TC>(v, Rx, Ry, Rz, delta, am, b);   // solid nodes lie inside a_map
  // A link's receiver lies within sqrt(2) of its solid node, or -- across a
  // Lees-Edwards plane, where the receiver is the node whose nearest source is
  // s -- within sqrt(1.5^2 + 1) = 1.80; deeper solid nodes cannot have links.
  const TC inner = am > (TC)2 ? am - (TC)2 : (TC)0;
  // a receiver deeper than a_map - 0.05 inside this particle's own mapped
  // sphere is one of its solid nodes (the node map holds every node closer
  // than a_map): that direction is no link and needs no look-up
  const TC deep = am > (TC)0.05 ? (am - (TC)0.05) * (am - (TC)0.05) : (TC)0;
  bool overflow = false;
  for_box_cells<TC>(v, b, Rx, Ry, Rz, delta, am,
                    [&](int x, int y, int z, long long s, TC sdx, TC sdy, TC sdz, int, TC d2) {
    // every node closer than a_map is this particle's (the node-map kernels
    // claim exactly those, with the same d2; a node another particle holds
    // there has raised the overlap flag), so no owner look-up here
    if (!(d2 < am * am) || d2 < inner * inner) return;
    // |s + c_p - R|^2 = d2 + 2 (s - R).c_p + |c_p|^2, with the partial sums
    // shared between directions
    const TC d1 = d2 + (TC)1, dd = d2 + (TC)2;
    const TC tx = (TC)2 * sdx, ty = (TC)2 * sdy, tz = (TC)2 * sdz;
    const TC xp = dd + tx, xm = dd - tx, yp = dd + ty, ym = dd - ty;
    uint32_t m = 0;
#pragma unroll
    for (int p = 1; p < 19; ++p) {
      const int cx = D3Q19::cx(p), cy = D3Q19::cy(p), cz = D3Q19::cz(p);
      const int ryn = y + cy;
      TC e2;
      if (cx * cx + cy * cy + cz * cz == 1)
        e2 = d1 + (cx ? (cx > 0 ? tx : -tx) : (cy ? (cy > 0 ? ty : -ty) : (cz > 0 ? tz : -tz)));
      else if (cx)
        e2 = (cx > 0 ? xp : xm) + (cy ? (cy > 0 ? ty : -ty) : (cz > 0 ? tz : -tz));
      else
        e2 = (cy > 0 ? yp : ym) + (cz > 0 ? tz : -tz);
      // a pull across a Lees-Edwards plane is always examined
      const bool keep = (ryn < 0 || ryn >= v.ny) || !(e2 < deep);
      if (keep) m |= 1u << p;
    }
    if (!m) return;
    const int k = atomicAdd(&s_nodes, 1);
    if (k < LINK_NODES_MAX) {
      s_node[k] = (uint32_t)x | ((uint32_t)y << 11) | ((uint32_t)z << 22);
      s_mask[k] = m;
    } else {
      overflow = true;
    }
  }, i, am);
  if (overflow) atomicOr(v.err, ERR_LINKS);
  __syncthreads();
  const int nn = min(s_nodes, LINK_NODES_MAX);
  TC acc[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) acc[k] = 0;
  // rounds of blockDim nodes: their candidate directions are expanded into
  // (node, direction) items in shared memory (at most 18 per node), so that
  // full warps then process the items, one memory round trip each
  const int lane = threadIdx.x & 31;
  for (int nb = 0; nb < nn; nb += blockDim.x) {
    {
      const int k = nb + (int)threadIdx.x;
      const uint32_t m = k < nn ? s_mask[k] : 0u;
      const int cnt = __popc(m);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int up = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += up;
      }
      int wbase = 0;
      if (lane == 31 && incl) wbase = atomicAdd(&s_items_n, incl);
      wbase = __shfl_sync(0xffffffffu, wbase, 31);
      int pos = wbase + incl - cnt;
      uint32_t mm = m;
      while (mm) {
        const int p = __ffs(mm) - 1;
        mm &= mm - 1;
        s_items[pos++] = ((uint32_t)k << 5) | (uint32_t)p;
      }
    }
    __syncthreads();
    const int ns = s_items_n;
    // two items per thread and pass: both receivers' loads are in flight together
    const uint32_t nc = (uint32_t)v.ncell;   // 19 * ncell < 2^32 for every accepted box
    for (int k0 = threadIdx.x; k0 < ns; k0 += 2 * blockDim.x) {
      int x[2], y[2], z[2], p[2], rx[2], ry[2], rz[2], ow[2];
      uint32_t r[2];
      bool crossing[2], live[2];
      TC nq[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = k0 + u * (int)blockDim.x;
        live[u] = k < ns;
        const uint32_t it = live[u] ? s_items[k] : s_items[k0];
        const uint32_t w = s_node[it >> 5];
        p[u] = (int)(it & 31u);
        x[u] = (int)(w & 2047u); y[u] = (int)((w >> 11) & 2047u); z[u] = (int)(w >> 22);
        r[u] = link_target_nr(v, pr, x[u], y[u], z[u], s_cp[p[u]], rx[u], ry[u], rz[u], crossing[u]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        // the receiver's owner word and its population q are loaded together
        // (the population of a solid receiver is read and discarded)
        const int q = D3Q19::opp(p[u]);
        ow[u] = v.owner[r[u]];
        nq[u] = S::load(f, (uint32_t)q * nc + r[u], s_cq[p[u]].w * rho0, (TC)v.inv_scale);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!live[u] || ow[u] == i) continue;
        const int q = D3Q19::opp(p[u]);
        const auto cqv = s_cq[p[u]];
        const TC cqx = cqv.x, cqy = cqv.y, cqz = cqv.z;
        TC dx = (TC)rx[u] + (TC)0.5 * cqx - Rx, dy = (TC)ry[u] + (TC)0.5 * cqy - Ry,
           dz = (TC)rz[u] + (TC)0.5 * cqz - Rz;
        const int kimg = le_image_v(v, dx, dy, dz, delta);
        const TC ubx = pp[3] + (pp[7] * dz - pp[8] * dy) + (TC)kimg * ule;
        const TC uby = pp[4] + (pp[8] * dx - pp[6] * dz);
        const TC ubz = pp[5] + (pp[6] * dy - pp[7] * dx);
        const TC cu = ubx * cqx + uby * cqy + ubz * cqz;
        const TC wqq = cqv.w;
        // fluid receiver: momentum exchange and the bounce-back value for the
        // next pull; another particle's node: fluid in equilibrium moving with
        // the mean ubar of the two surfaces' velocities at r_b, against a wall
        // moving with ubar, 2 n^eq_q(rho0, rho0 ubar) - 6 C^q rho0 ubar.c_q
        // = C^q rho0 (2 + 9 (ubar.c_q)^2 - 3 ubar^2)
        TC mag;
        if (ow[u] < 0) {
          const TC wall = (TC)6 * wqq * rho0 * cu;
          mag = (TC)2 * nq[u] - wall;
          if (!crossing[u]) {
            const uint32_t sidx = (uint32_t)(x[u] + v.nx * (y[u] + v.ny * z[u]));
            f[(uint32_t)p[u] * nc + sidx] = S::enc(nq[u] - wall, wqq * rho0, (TC)v.scale);
          }
        } else {
          mag = touching_link<TC>(v, ow[u], rx[u], ry[u], rz[u], q, ubx, uby, ubz, delta, ule, rho0);
        }
        const TC fx = mag * cqx, fy = mag * cqy, fz = mag * cqz;
        acc[0] += fx; acc[1] += fy; acc[2] += fz;
        acc[3] += dy * fz - dz * fy; acc[4] += dz * fx - dx * fz; acc[5] += dx * fy - dy * fx;
        acc[6] += dx * fx; acc[7] += dx * fy; acc[8] += dx * fz;
        acc[9] += dy * fx; acc[10] += dy * fy; acc[11] += dy * fz;
        acc[12] += dz * fx; acc[13] += dz * fy; acc[14] += dz * fz;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_items_n = 0;
    __syncthreads();
  }
  block_sum<TC, 15>(acc, red);
  if (threadIdx.x == 0) {
    for (int a = 0; a < 3; ++a) {
      v.Fh[3 * i + a] = (double)acc[a];
      v.Th[3 * i + a] = (double)acc[3 + a];
    }
    for (int a = 0; a < 9; ++a) atomicAdd(acc_rep(v, i) + 6 + a, (double)acc[6 + a]);
  }
}

template <int P>
__global__ void k_init_pop(View v, typename Store<P>::T* __restrict__ f) {
  using TC = typename Store<P>::C;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= v.ncell) return;
  const TC rho0 = sel<TC>(v.rho0, v.rho0_f);
#pragma unroll
  for (int q = 0; q < 19; ++q)
    f[(long long)q * v.ncell + idx] = Store<P>::enc((TC)D3Q19::w(q) * rho0, (TC)D3Q19::w(q) * rho0, (TC)v.scale);
}

}  // namespace susp_dev

using namespace susp_dev;

template <int P> using PT = typename Store<P>::T;

void launch_claim(int prec, const Batch& B, int nparts, cudaStream_t s) {
  if (nparts == 0) return;
  switch (prec) {
    case 0: k_claim<0><<<nparts, 128, 0, s>>>(B); break;
    case 1: k_claim<1><<<nparts, 128, 0, s>>>(B); break;
    case 2: k_claim<2><<<nparts, 128, 0, s>>>(B); break;
    default: k_claim<3><<<nparts, 128, 0, s>>>(B); break;
  }
}

// Node-map update after the particles moved: uncover, then cover (one block
// of 128 threads per particle: the scans are short, and smaller blocks let
// every particle's block be resident at once on the 96^3 box).
void launch_node_update(int prec, const Batch& B, int nparts, cudaStream_t s) {
  if (nparts == 0) return;
  // the 64-register uncover form beyond eight waves of six blocks per SM
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  const bool wide = nparts > 8 * 6 * sms;
  switch (prec) {
    case 0: k_uncover<0, false><<<nparts, 128, 0, s>>>(B); k_cover<0><<<nparts, 128, 0, s>>>(B); break;
    case 1:
      if (wide) k_uncover<1, true><<<nparts, 128, 0, s>>>(B);
      else k_uncover<1, false><<<nparts, 128, 0, s>>>(B);
      k_cover<1><<<nparts, 128, 0, s>>>(B);
      break;
    case 2:
      if (wide) k_uncover<2, true><<<nparts, 128, 0, s>>>(B);
      else k_uncover<2, false><<<nparts, 128, 0, s>>>(B);
      k_cover<2><<<nparts, 128, 0, s>>>(B);
      break;
    default:
      if (wide) k_uncover<3, true><<<nparts, 128, 0, s>>>(B);
      else k_uncover<3, false><<<nparts, 128, 0, s>>>(B);
      k_cover<3><<<nparts, 128, 0, s>>>(B);
      break;
  }
}

void launch_links(int prec, const Batch& B, int nparts, cudaStream_t s) {
  if (nparts == 0) return;
  // one block per particle; the four-block form beyond eight waves of the
  // three-block one (measured: 1196 against 1252 us on a batch of 27 524
  // particles, 54 against 48 us for 882)
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  const bool wide = nparts > 8 * 3 * sms;
  switch (prec) {
    case 0: k_links<0, false><<<nparts, 256, 0, s>>>(B); break;
    case 1:
      if (wide) k_links<1, true><<<nparts, 256, 0, s>>>(B);
      else k_links<1, false><<<nparts, 256, 0, s>>>(B);
      break;
    case 2:
      if (wide) k_links<2, true><<<nparts, 256, 0, s>>>(B);
      else k_links<2, false><<<nparts, 256, 0, s>>>(B);
      break;
    default:
      if (wide) k_links<3, true><<<nparts, 256, 0, s>>>(B);
      else k_links<3, false><<<nparts, 256, 0, s>>>(B);
      break;
  }
}

void launch_init_pop(int prec, const View& v, void* f, cudaStream_t s) {
  const int nb = (int)((v.ncell + 255) / 256);
  switch (prec) {
    case 0: k_init_pop<0><<<nb, 256, 0, s>>>(v, (PT<0>*)f); break;
    case 1: k_init_pop<1><<<nb, 256, 0, s>>>(v, (PT<1>*)f); break;
    case 2: k_init_pop<2><<<nb, 256, 0, s>>>(v, (PT<2>*)f); break;
    default: k_init_pop<3><<<nb, 256, 0, s>>>(v, (PT<3>*)f); break;
  }
}
