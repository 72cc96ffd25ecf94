// api.cu — C ABI (include/susp.h): workspace layout, step sequencing, the
// per-step stress / protocol finalisation kernel and host-side read-back.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/susp.h"
#include "susp_dev.cuh"

using namespace susp_dev;

// launchers defined in the other translation units
void launch_plane_moments(int prec, const View& v, const void* fin, cudaStream_t s);
void launch_collide_stream(int prec, const View& v, const void* fin, void* fout, cudaStream_t s);
int lb_blocks(int nx, int ny, int nz);
int lb_grid_blocks(int prec, int nx, int ny, int nz);
void launch_claim(int prec, const View& v, cudaStream_t s);
void launch_node_update(int prec, const View& v, void* f, cudaStream_t s);
void launch_links(int prec, const View& v, const void* f, cudaStream_t s);
void launch_init_pop(int prec, const View& v, void* f, cudaStream_t s);
void launch_write_plb(const View& v, int plb_double, cudaStream_t s);
void launch_dem_substep(const View& v, int parity, int sub, int plb_double, cudaStream_t s);

namespace {

thread_local std::string g_err = "";

susp_status fail(susp_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

const int HSLOTS = 16;        // tangential springs per particle (partners with larger index)
const int FIN_BLOCKS = 32;    // blocks of the per-step finalisation
const int FIN_VALS = 40;      // 6 visc, 9 stresslet, 9 contact, 1 contacts, 9 repulsive
const double KPI = 3.14159265358979323846;

size_t esize(int prec) { return prec == 0 ? 8 : (prec == 1 ? 4 : 2); }
size_t csize(int prec) { return prec == 0 ? 8 : 4; }
size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t fa, fb, mask, owner, pm, visc;
  size_t R, U, W, rad, amap, mass, inert, imass, iinert, plb, Fh, Th, Fcov, Tcov, Fp, Tp;
  size_t slet, cvir, rvir, ncont, links, loff, lcap, lcnt;
  size_t cstart, ccnt, cids, pcell;
  size_t hc0, hp0, hv0, hc1, hp1, hv1;
  size_t sums, hist, counters, proto, err, finp, finc;
  size_t total;
  long long nlinks;
  int ncx, ncy, ncz, brute, ncells;
  double csx, csy, csz, hrange;
};

bool valid(const susp_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return false; }
  if (p->nx < 4 || p->ny < 4 || p->nz < 4) { why = "lattice dims must be >= 4"; return false; }
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 27)) { why = "lattice larger than 2^27 nodes"; return false; }
  if (!(p->tau > 0.5)) { why = "tau must exceed 1/2"; return false; }
  if (!(p->rho0 > 0.0)) { why = "rho0 must be positive"; return false; }
  if (p->n < 0) { why = "n < 0"; return false; }
  if (p->n > 0 && (!p->radius || !p->pos)) { why = "radius / pos missing"; return false; }
  if (p->prec < SUSP_FP64 || p->prec > SUSP_BF16_DEV) { why = "bad precision"; return false; }
  if (p->n > 0) {
    if (!(p->rho_p > 0.0) || !(p->kn > 0.0) || !(p->kt_ratio > 0.0) || !(p->mu >= 0.0)) {
      why = "particle parameters must be positive"; return false;
    }
    if (!(p->a_map_ratio > 0.0 && p->a_map_ratio <= 1.0)) { why = "a_map_ratio in (0, 1]"; return false; }
    for (int i = 0; i < p->n; ++i) {
      if (!(p->radius[i] > 0.0)) { why = "radius must be positive"; return false; }
      double am = p->a_map_ratio * p->radius[i] + 1.0;
      if (2 * am + 1 >= p->nx || 2 * am + 1 >= p->ny || 2 * am + 1 >= p->nz) {
        why = "particle too large for the box"; return false;
      }
    }
  }
  return true;
}

double hrange_of(const susp_params* p) {
  double h = 0.0;
  if (p->lub_cut > 0.0) h = p->lub_cut;
  if (p->F0 > 0.0 && 10.0 * p->debye > h) h = 10.0 * p->debye;
  return h;
}

void make_layout(const susp_params* p, Layout& L) {
  const long long nc = (long long)p->nx * p->ny * p->nz;
  const int n = p->n, nn = n > 0 ? n : 1;
  const int prec = p->prec;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
  L.fa = take(19 * nc * esize(prec));
  L.fb = take(19 * nc * esize(prec));
  L.mask = take(4 * nc);
  L.owner = take(4 * nc);
  L.pm = take(2ULL * p->nx * p->nz * 4 * csize(prec));
  L.visc = take(6 * 8 * (size_t)lb_blocks(p->nx, p->ny, p->nz));
  L.R = take(24 * nn); L.U = take(24 * nn); L.W = take(24 * nn);
  L.rad = take(8 * nn); L.amap = take(8 * nn); L.mass = take(8 * nn); L.inert = take(8 * nn);
  L.imass = take(8 * nn); L.iinert = take(8 * nn);
  L.plb = take(12 * csize(prec) * nn);
  L.Fh = take(24 * nn); L.Th = take(24 * nn); L.Fcov = take(24 * nn); L.Tcov = take(24 * nn);
  L.Fp = take(24 * nn); L.Tp = take(24 * nn);
  L.slet = take(72 * nn); L.cvir = take(72 * nn); L.rvir = take(72 * nn); L.ncont = take(4 * nn);
  long long nl = 0;
  for (int i = 0; i < n; ++i) {
    double am = p->a_map_ratio * p->radius[i] + 1.0;
    nl += (long long)ceil(6.0 * 4.0 * KPI * am * am) + 64;
  }
  L.nlinks = nl;
  L.links = take(4 * (nl > 0 ? nl : 1));
  L.loff = take(4 * nn); L.lcap = take(4 * nn); L.lcnt = take(4 * nn);
  // cell list geometry
  double amax = 0.0;
  for (int i = 0; i < n; ++i) amax = std::max(amax, p->radius[i]);
  L.hrange = hrange_of(p);
  const double cmin = 2.0 * amax + L.hrange + 1.0;
  int ncx = (int)floor(p->nx / cmin), ncy = (int)floor(p->ny / cmin), ncz = (int)floor(p->nz / cmin);
  if (ncx < 3 || ncy < 3) { ncx = ncy = ncz = 1; L.brute = 1; }
  else { L.brute = 0; if (ncz < 1) ncz = 1; }
  L.ncx = ncx; L.ncy = ncy; L.ncz = ncz;
  L.ncells = ncx * ncy * ncz;
  L.csx = (double)p->nx / ncx; L.csy = (double)p->ny / ncy; L.csz = (double)p->nz / ncz;
  L.cstart = take(4 * (L.ncells + 1)); L.ccnt = take(4 * L.ncells);
  L.cids = take(4 * nn); L.pcell = take(4 * nn);
  L.hc0 = take(4 * nn); L.hp0 = take(4 * (size_t)nn * HSLOTS); L.hv0 = take(24 * (size_t)nn * HSLOTS);
  L.hc1 = take(4 * nn); L.hp1 = take(4 * (size_t)nn * HSLOTS); L.hv1 = take(24 * (size_t)nn * HSLOTS);
  L.sums = take(8 * 72);
  int nb = p->nbins > 0 ? p->nbins : 36;
  L.hist = take(8 * 3 * nb);
  L.counters = take(8 * 4);
  L.proto = take(sizeof(Proto));
  L.err = take(4);
  L.finp = take(8 * FIN_VALS * FIN_BLOCKS);
  L.finc = take(4);
  L.total = o;
}

// ------------------------------------------------------------ device kernels

__device__ void proto_derive(Proto& s, int nx) {
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

__device__ void kahan_le(double& delta, double& comp, double inc, int nx) {
  const double y = inc - comp;
  const double t = delta + y;
  comp = (t - delta) - y;
  delta = t;
  if (delta >= nx) delta -= nx;
  if (delta < 0.0) delta += nx;
}

// Set a new shear protocol at the current step (keeps t and Delta_t).
__global__ void k_proto_set(Proto* pp, int nx, int kind, double rate, double gamma0, double omega,
                            double theta) {
  Proto s = *pp;
  s.kind = kind; s.rate = rate; s.gamma0 = gamma0; s.omega = omega; s.theta = theta;
  s.ule = proto_increment(s, s.t);
  s.delta_n = s.delta; s.delta_nc = s.delta_c;
  kahan_le(s.delta_n, s.delta_nc, s.ule, nx);
  s.ule_n = proto_increment(s, s.t + 1);
  proto_derive(s, nx);
  *pp = s;
}

// End of step t: reduce the per-block / per-particle stress partials, add
// them to the compensated time sums, then advance the protocol to t+1.
// FIN_BLOCKS blocks each reduce a slice into fin_part; the last block to
// finish sums the slices in block order, so the result is deterministic.
__global__ void __launch_bounds__(256) k_finalize(View v, double* fin_part, unsigned* fin_count) {
  __shared__ double red[32 * 37];
  __shared__ bool last;
  double acc[37];
  for (int k = 0; k < 37; ++k) acc[k] = 0.0;
  const int G = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = G * blockDim.x;
  for (int b = tid; b < v.nblk_lb; b += nthr)
    for (int k = 0; k < 6; ++k) acc[k] += v.visc_part[6LL * b + k];
  for (int i = tid; i < v.n; i += nthr) {
    for (int k = 0; k < 9; ++k) {
      acc[6 + k] += v.slet_part[9 * i + k];
      acc[15 + k] += v.cvir_part[9 * i + k];
      acc[25 + k] += v.rvir_part[9 * i + k];
    }
    acc[24] += v.ncont_part[i];
  }
  block_sum<double, 37>(acc, red);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 37; ++k) fin_part[FIN_VALS * blockIdx.x + k] = acc[k];
    __threadfence();
    last = (atomicAdd(fin_count, 1u) == (unsigned)G - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // column k of the slices, summed in block order by thread k
  __shared__ double tot[37];
  if (threadIdx.x < 37) {
    double t = 0.0;
    for (int b = 0; b < G; ++b) t += ((volatile double*)fin_part)[FIN_VALS * b + threadIdx.x];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  *fin_count = 0u;
  // visc partials: xx yy zz xy xz yz -> full 3x3
  const double vs[9] = {tot[0], tot[3], tot[4], tot[3], tot[1], tot[5], tot[4], tot[5], tot[2]};
  double* S = v.sums;
  double* Cc = v.sums + 36;
  for (int k = 0; k < 36; ++k) {
    double x;
    if (k < 9) x = vs[k];
    else if (k < 18) x = tot[6 + (k - 9)];
    else if (k < 27) x = v.move ? tot[15 + (k - 18)] : 0.0;
    else x = v.move ? tot[25 + (k - 27)] : 0.0;
    const double y = x - Cc[k];
    const double t = S[k] + y;
    Cc[k] = (t - S[k]) - y;
    S[k] = t;
  }
  v.counters[0] += 1ULL;
  if (v.move) v.counters[1] += (unsigned long long)(tot[24] + 0.5);
  // protocol: t -> t+1
  Proto s = *v.proto;
  s.t += 1;
  s.delta = s.delta_n; s.delta_c = s.delta_nc; s.ule = s.ule_n;
  s.delta_n = s.delta; s.delta_nc = s.delta_c;
  kahan_le(s.delta_n, s.delta_nc, s.ule, v.nx);
  s.ule_n = proto_increment(s, s.t + 1);
  proto_derive(s, v.nx);
  *v.proto = s;
}

}  // namespace

// ------------------------------------------------------------ handle

struct susp {
  susp_params p;
  int prec;
  Layout L;
  View v;
  char* ws;
  void* fin;
  void* fout;
  cudaStream_t stream;
  int parity;
  bool have_shear;
  susp_shear shear;
  std::vector<double> radius;
  double scale;
  // instrumentation
  bool prof;
  int prof_n;
  std::vector<cudaEvent_t> ev;
};

static const int PROF_MAX = 4096;

static susp_status cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(SUSP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return SUSP_OK;
}

static susp_status device_status(susp* h) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(SUSP_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
  int err = 0;
  e = cudaMemcpy(&err, h->v.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(SUSP_ECUDA, std::string("read error flag: ") + cudaGetErrorString(e));
  if (err & ERR_OVERLAP) return fail(SUSP_EOVERLAP, "two mapped spheres claimed one node");
  if (err & ERR_UNSTABLE) return fail(SUSP_EUNSTABLE, "non-positive density or particle speed >= 0.5");
  if (err & ERR_LINKS) return fail(SUSP_ENOMEM, "boundary-link table full");
  if (err & ERR_PAIRS) return fail(SUSP_ENOMEM, "tangential-spring table full");
  return SUSP_OK;
}

static void refresh_links(susp* h) {
  launch_links(h->prec, h->v, h->fin, h->stream);
}

void susp_set_last_error(const char* msg) { g_err = msg; }

extern "C" {

const char* susp_last_error(void) { return g_err.c_str(); }

size_t susp_workspace_bytes(const susp_params* p) {
  std::string why;
  if (!valid(p, why)) { g_err = why; return 0; }
  Layout L;
  make_layout(p, L);
  return L.total;
}

susp_status susp_create(const susp_params* p, void* dev_workspace, size_t bytes, void* cuda_stream,
                        susp** out) {
  if (out) *out = nullptr;
  std::string why;
  if (!out) return fail(SUSP_EINVAL, "out is NULL");
  if (!valid(p, why)) return fail(SUSP_EINVAL, why);
  if (!dev_workspace || ((uintptr_t)dev_workspace & 255)) return fail(SUSP_EINVAL, "workspace NULL or not 256-byte aligned");
  Layout L;
  make_layout(p, L);
  if (bytes < L.total) return fail(SUSP_ENOMEM, "workspace smaller than susp_workspace_bytes()");
  susp* h = new susp();
  h->p = *p;
  h->p.radius = h->p.pos = h->p.vel = h->p.omega = nullptr;
  h->prec = (int)p->prec;
  h->L = L;
  h->ws = (char*)dev_workspace;
  h->stream = (cudaStream_t)cuda_stream;
  h->parity = 0;
  h->have_shear = false;
  h->radius.assign(p->radius, p->radius + p->n);
  h->prof = false;
  h->prof_n = 0;
  h->scale = p->prec == SUSP_FP16_DEV ? 4096.0 : 1.0;
  char* w = h->ws;
  View& v = h->v;
  memset(&v, 0, sizeof(View));
  const int n = p->n;
  v.nx = p->nx; v.ny = p->ny; v.nz = p->nz;
  v.ncell = (long long)p->nx * p->ny * p->nz;
  v.tau = p->tau; v.rho0 = p->rho0;
  for (int a = 0; a < 3; ++a) { v.g[a] = p->body_force[a]; v.g_f[a] = (float)p->body_force[a]; }
  v.scale = (float)h->scale; v.inv_scale = (float)(1.0 / h->scale);
  v.omega_d = 1.0 / p->tau; v.vf_d = -(1.0 - 0.5 / p->tau);
  v.omega_f = (float)v.omega_d; v.vf_f = (float)v.vf_d; v.rho0_f = (float)p->rho0;
  v.inv_nx_d = 1.0 / p->nx; v.inv_ny_d = 1.0 / p->ny; v.inv_nz_d = 1.0 / p->nz;
  v.inv_nx_f = (float)v.inv_nx_d; v.inv_ny_f = (float)v.inv_ny_d; v.inv_nz_f = (float)v.inv_nz_d;
  v.mask = (uint32_t*)(w + L.mask); v.owner = (int*)(w + L.owner);
  v.plane_mom = w + L.pm; v.visc_part = (double*)(w + L.visc); v.nblk_lb = lb_grid_blocks((int)p->prec, p->nx, p->ny, p->nz);
  v.n = n;
  v.R = (double*)(w + L.R); v.U = (double*)(w + L.U); v.W = (double*)(w + L.W);
  v.rad = (double*)(w + L.rad); v.amap = (double*)(w + L.amap);
  v.mass = (double*)(w + L.mass); v.inert = (double*)(w + L.inert);
  v.inv_m = (double*)(w + L.imass); v.inv_I = (double*)(w + L.iinert);
  v.plb = w + L.plb;
  v.Fh = (double*)(w + L.Fh); v.Th = (double*)(w + L.Th);
  v.Fcov = (double*)(w + L.Fcov); v.Tcov = (double*)(w + L.Tcov);
  v.Fp = (double*)(w + L.Fp); v.Tp = (double*)(w + L.Tp);
  v.slet_part = (double*)(w + L.slet); v.cvir_part = (double*)(w + L.cvir);
  v.rvir_part = (double*)(w + L.rvir); v.ncont_part = (int*)(w + L.ncont);
  v.links = (uint32_t*)(w + L.links); v.link_off = (int*)(w + L.loff);
  v.link_cap = (int*)(w + L.lcap); v.link_cnt = (int*)(w + L.lcnt);
  v.ncx = L.ncx; v.ncy = L.ncy; v.ncz = L.ncz; v.brute = L.brute; v.ncells = L.ncells;
  v.csx = L.csx; v.csy = L.csy; v.csz = L.csz;
  v.inv_csx = 1.0 / L.csx; v.inv_csy = 1.0 / L.csy; v.inv_csz = 1.0 / L.csz;
  v.cell_start = (int*)(w + L.cstart); v.cell_cnt = (int*)(w + L.ccnt);
  v.cell_ids = (int*)(w + L.cids); v.pcell = (int*)(w + L.pcell);
  v.K = HSLOTS;
  v.hcnt0 = (int*)(w + L.hc0); v.hpart0 = (int*)(w + L.hp0); v.hval0 = (double*)(w + L.hv0);
  v.hcnt1 = (int*)(w + L.hc1); v.hpart1 = (int*)(w + L.hp1); v.hval1 = (double*)(w + L.hv1);
  // physics
  double m0 = 0.0;
  std::vector<double> mass(n), inert(n), amap(n);
  for (int i = 0; i < n; ++i) {
    double a = p->radius[i];
    mass[i] = p->rho_p * 4.0 / 3.0 * KPI * a * a * a;
    inert[i] = 0.4 * mass[i] * a * a;
    amap[i] = p->a_map_ratio * a;
    m0 += mass[i];
  }
  if (n > 0) m0 /= n;
  v.mu = p->mu; v.kn = p->kn; v.kt = p->kt_ratio * p->kn;
  v.eta_n = p->eta_n >= 0.0 ? p->eta_n : sqrt(m0 * p->kn);
  v.F0 = p->F0; v.debye = p->debye; v.lub_delta = p->lub_delta; v.lub_cut = p->lub_cut;
  v.eta0 = p->rho0 * (p->tau - 0.5) / 3.0;
  v.hrange = L.hrange;
  v.quasi2d = p->quasi2d; v.move = p->move_particles;
  v.nbins = p->nbins > 0 ? p->nbins : 36;
  if (p->dem_substeps > 0) v.nsub = p->dem_substeps;
  else if (n == 0) v.nsub = 1;
  else {
    double mmin = 1e300, amin = 1e300;
    for (int i = 0; i < n; ++i) { mmin = std::min(mmin, mass[i]); amin = std::min(amin, p->radius[i]); }
    double om = sqrt(2.0 * p->kn / mmin);
    double zeta = (p->lub_cut > 0.0 && p->lub_delta > 0.0) ? v.eta0 * 1.5 * KPI * amin * amin / p->lub_delta : 0.0;
    double c = 2.0 * (v.eta_n + zeta) / mmin;
    v.nsub = std::max(1, (int)ceil(std::max(om, c)));
  }
  v.sums = (double*)(w + L.sums); v.hist = (double*)(w + L.hist);
  v.counters = (unsigned long long*)(w + L.counters);
  v.proto = (Proto*)(w + L.proto); v.err = (int*)(w + L.err);
  h->fin = w + L.fa;
  h->fout = w + L.fb;

  cudaStream_t s = h->stream;
  susp_status st = SUSP_OK;
  // zero everything past the populations, then fill
  st = cuda_check(cudaMemsetAsync(w + L.mask, 0, L.total - L.mask, s), "memset workspace");
  if (st) { delete h; return st; }
  cudaMemsetAsync(v.owner, 0xff, 4 * v.ncell, s);
  if (n > 0) {
    std::vector<double> zeros(3 * n, 0.0);
    std::vector<int> off(n), cap(n);
    long long acc = 0;
    for (int i = 0; i < n; ++i) {
      double am = amap[i] + 1.0;
      cap[i] = (int)ceil(6.0 * 4.0 * KPI * am * am) + 64;
      off[i] = (int)acc;
      acc += cap[i];
    }
    std::vector<double> R(p->pos, p->pos + 3 * n);
    cudaMemcpyAsync(v.R, R.data(), 24 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.U, p->vel ? p->vel : zeros.data(), 24 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.W, p->omega ? p->omega : zeros.data(), 24 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.rad, p->radius, 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.amap, amap.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.mass, mass.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.inert, inert.data(), 8 * n, cudaMemcpyHostToDevice, s);
    std::vector<double> im(n), iI(n);
    for (int i = 0; i < n; ++i) { im[i] = 1.0 / mass[i]; iI[i] = 1.0 / inert[i]; }
    cudaMemcpyAsync(v.inv_m, im.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.inv_I, iI.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.link_off, off.data(), 4 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.link_cap, cap.data(), 4 * n, cudaMemcpyHostToDevice, s);
    // synchronous copies above read pageable host memory; wait before the vectors go away
    st = cuda_check(cudaStreamSynchronize(s), "upload particles");
    if (st) { delete h; return st; }
  }
  Proto pr;
  memset(&pr, 0, sizeof pr);
  pr.ny = p->ny;
  cudaMemcpyAsync(v.proto, &pr, sizeof pr, cudaMemcpyHostToDevice, s);
  k_proto_set<<<1, 1, 0, s>>>(v.proto, v.nx, 0, 0.0, 0.0, 0.0, 0.0);
  launch_init_pop(h->prec, v, h->fin, s);
  launch_init_pop(h->prec, v, h->fout, s);
  launch_write_plb(v, h->prec == 0, s);
  launch_claim(h->prec, v, s);
  refresh_links(h);
  st = cuda_check(cudaGetLastError(), "launch");
  if (st) { delete h; return st; }
  st = device_status(h);
  if (st) { delete h; return st; }
  *out = h;
  return SUSP_OK;
}

susp_status susp_step(susp* h, int nsteps, const susp_shear* sh) {
  if (!h || !sh || nsteps < 0) return fail(SUSP_EINVAL, "bad argument to susp_step");
  if (sh->kind != 0 && sh->kind != 1) return fail(SUSP_EINVAL, "shear kind must be 0 or 1");
  cudaStream_t s = h->stream;
  View& v = h->v;
  if (!h->have_shear || memcmp(&h->shear, sh, sizeof(susp_shear)) != 0) {
    k_proto_set<<<1, 1, 0, s>>>(v.proto, v.nx, sh->kind, sh->rate, sh->gamma0, sh->omega, sh->theta);
    refresh_links(h);   // the image velocity of the boundary links changed
    h->shear = *sh;
    h->have_shear = true;
  }
  for (int it = 0; it < nsteps; ++it) {
    launch_plane_moments(h->prec, v, h->fin, s);
    const bool timed = h->prof && h->prof_n < PROF_MAX;
    if (timed) cudaEventRecord(h->ev[2 * h->prof_n], s);
    launch_collide_stream(h->prec, v, h->fin, h->fout, s);
    if (timed) { cudaEventRecord(h->ev[2 * h->prof_n + 1], s); ++h->prof_n; }
    if (v.move && v.n > 0) {
      for (int sub = 0; sub < v.nsub; ++sub) {
        launch_dem_substep(v, h->parity, sub, h->prec == 0, s);
        h->parity ^= 1;
      }
    }
    k_finalize<<<FIN_BLOCKS, 256, 0, s>>>(v, (double*)(h->ws + h->L.finp), (unsigned*)(h->ws + h->L.finc));
    launch_node_update(h->prec, v, h->fout, s);
    launch_links(h->prec, v, h->fout, s);
    std::swap(h->fin, h->fout);
  }
  return cuda_check(cudaGetLastError(), "launch");
}

susp_status susp_stress_reset(susp* h) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->v.sums, 0, 8 * 72, s);
  cudaMemsetAsync(h->v.hist, 0, 8 * 3 * h->v.nbins, s);
  cudaMemsetAsync(h->v.counters, 0, 8 * 2, s);
  return cuda_check(cudaGetLastError(), "stress reset");
}

susp_status susp_stress(susp* h, susp_stress_kind kind, double out[9], double* hist, int nbins) {
  if (!h || !out) return fail(SUSP_EINVAL, "NULL argument");
  susp_status st = device_status(h);
  if (st) return st;
  double sums[72];
  unsigned long long cnt[2];
  std::vector<double> hs(3 * h->v.nbins);
  cudaMemcpy(sums, h->v.sums, sizeof sums, cudaMemcpyDeviceToHost);
  cudaMemcpy(cnt, h->v.counters, sizeof cnt, cudaMemcpyDeviceToHost);
  cudaMemcpy(hs.data(), h->v.hist, 8 * hs.size(), cudaMemcpyDeviceToHost);
  st = cuda_check(cudaGetLastError(), "read stress");
  if (st) return st;
  if (hist && nbins == h->v.nbins) memcpy(hist, hs.data(), 8 * hs.size());
  for (int k = 0; k < 9; ++k) out[k] = 0.0;
  if (cnt[0] == 0) return SUSP_OK;
  const double V = (double)h->v.nx * h->v.ny * h->v.nz;
  const double norm = 1.0 / (V * (double)cnt[0]);
  double visc[9], cont[9], rep[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const int k = 3 * a + b, kt = 3 * b + a;
      visc[k] = norm * (sums[k] + 0.5 * (sums[9 + k] + sums[9 + kt]));
      cont[k] = -norm * sums[18 + k];
      rep[k] = -norm * sums[27 + k];
    }
  switch (kind) {
    case SUSP_STRESS_VISCOUS: memcpy(out, visc, sizeof visc); break;
    case SUSP_STRESS_CONTACT: memcpy(out, cont, sizeof cont); break;
    case SUSP_STRESS_REPULSIVE: memcpy(out, rep, sizeof rep); break;
    case SUSP_STRESS_TOTAL:
      for (int k = 0; k < 9; ++k) out[k] = visc[k] + cont[k] + rep[k];
      break;
    case SUSP_STRESS_ANGULAR: {
      // Eq. 26 (monolayer) or Eq. 27 from the histogram, midpoint rule over
      // the bins, rho normalised over [0, pi) (Eq. 23).
      const int nb = h->v.nbins;
      double nc = 0.0, sfn = 0.0;
      for (int b = 0; b < nb; ++b) { nc += hs[3 * b]; sfn += hs[3 * b + 1]; }
      if (!(nc > 0.0) || h->v.n == 0) break;
      double asum = 0.0, vol = 0.0, area = 0.0;
      for (double a : h->radius) { asum += a; vol += 4.0 / 3.0 * KPI * a * a * a; area += KPI * a * a; }
      const double amean = asum / h->v.n;
      const double Z = 2.0 * (double)cnt[1] / ((double)h->v.n * (double)cnt[0]);
      const double fmean = sfn / nc;
      const double dth = KPI / nb;
      double pref;
      if (h->v.quasi2d) pref = (area / ((double)h->v.nx * h->v.ny)) * Z * fmean / (KPI * amean);
      else pref = 3.0 * (vol / V) * Z * fmean / (2.0 * KPI * amean * amean);
      for (int b = 0; b < nb; ++b) {
        const double th = (b + 0.5) * dth;
        const double zn = hs[3 * b + 1] / (nc * dth * fmean), zt = hs[3 * b + 2] / (nc * dth * fmean);
        const double nv[2] = {cos(th), sin(th)}, tv[2] = {-sin(th), cos(th)};
        for (int al = 0; al < 2; ++al)
          for (int be = 0; be < 2; ++be) out[3 * al + be] += pref * (zn * nv[al] - zt * tv[al]) * nv[be] * dth;
      }
      break;
    }
    default: return fail(SUSP_EINVAL, "bad stress kind");
  }
  return SUSP_OK;
}

susp_status susp_get_particles(susp* h, double* pos, double* vel, double* omega) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  susp_status st = device_status(h);
  if (st) return st;
  const size_t b = 24 * (size_t)h->v.n;
  if (b == 0) return SUSP_OK;
  if (pos) cudaMemcpy(pos, h->v.R, b, cudaMemcpyDeviceToHost);
  if (vel) cudaMemcpy(vel, h->v.U, b, cudaMemcpyDeviceToHost);
  if (omega) cudaMemcpy(omega, h->v.W, b, cudaMemcpyDeviceToHost);
  return cuda_check(cudaGetLastError(), "read particles");
}

susp_status susp_get_hydro(susp* h, double* force, double* torque) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  susp_status st = device_status(h);
  if (st) return st;
  const size_t b = 24 * (size_t)h->v.n;
  if (b == 0) return SUSP_OK;
  if (force) cudaMemcpy(force, h->v.Fh, b, cudaMemcpyDeviceToHost);
  if (torque) cudaMemcpy(torque, h->v.Th, b, cudaMemcpyDeviceToHost);
  return cuda_check(cudaGetLastError(), "read hydro");
}

static inline float half_to_float(uint16_t hbits) {
  const uint32_t sign = (uint32_t)(hbits & 0x8000u) << 16;
  uint32_t exp = (hbits >> 10) & 0x1fu, man = hbits & 0x3ffu;
  uint32_t bits;
  if (exp == 0) {
    if (man == 0) bits = sign;
    else {
      exp = 127 - 15 + 1;
      while (!(man & 0x400u)) { man <<= 1; --exp; }
      man &= 0x3ffu;
      bits = sign | (exp << 23) | (man << 13);
    }
  } else if (exp == 31) bits = sign | 0x7f800000u | (man << 13);
  else bits = sign | ((exp + 127 - 15) << 23) | (man << 13);
  float f;
  memcpy(&f, &bits, 4);
  return f;
}

static inline uint16_t float_to_half(float f) {
  uint32_t x;
  memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u;
  const int exp = (int)((x >> 23) & 0xffu) - 127 + 15;
  uint32_t man = x & 0x7fffffu;
  if (((x >> 23) & 0xffu) == 0xffu) return (uint16_t)(sign | 0x7c00u | (man ? 0x200u : 0));
  if (exp >= 31) return (uint16_t)(sign | 0x7c00u);
  if (exp <= 0) {
    if (exp < -10) return (uint16_t)sign;
    man |= 0x800000u;
    const int shift = 14 - exp;
    uint32_t hm = man >> shift;
    const uint32_t rem = man & ((1u << shift) - 1), halfway = 1u << (shift - 1);
    if (rem > halfway || (rem == halfway && (hm & 1u))) ++hm;
    return (uint16_t)(sign | hm);
  }
  uint32_t hm = man >> 13;
  const uint32_t rem = man & 0x1fffu;
  uint32_t out = sign | ((uint32_t)exp << 10) | hm;
  if (rem > 0x1000u || (rem == 0x1000u && (hm & 1u))) ++out;
  return (uint16_t)out;
}

static inline float bf16_to_float(uint16_t b) {
  uint32_t x = (uint32_t)b << 16;
  float f;
  memcpy(&f, &x, 4);
  return f;
}
static inline uint16_t float_to_bf16(float f) {
  uint32_t x;
  memcpy(&x, &f, 4);
  if ((x & 0x7f800000u) == 0x7f800000u) return (uint16_t)((x >> 16) | ((x & 0xffffu) ? 0x40u : 0));
  const uint32_t lsb = (x >> 16) & 1u;
  x += 0x7fffu + lsb;
  return (uint16_t)(x >> 16);
}

static const double WQ[19] = {1.0 / 3, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

susp_status susp_get_populations(susp* h, double* f) {
  if (!h || !f) return fail(SUSP_EINVAL, "NULL argument");
  susp_status st = device_status(h);
  if (st) return st;
  const long long nc = h->v.ncell, tot = 19 * nc;
  const size_t es = esize(h->prec);
  std::vector<char> raw(tot * es);
  st = cuda_check(cudaMemcpy(raw.data(), h->fin, raw.size(), cudaMemcpyDeviceToHost), "read populations");
  if (st) return st;
  const double inv = 1.0 / h->scale;
  for (long long k = 0; k < tot; ++k) {
    const int q = (int)(k / nc);
    const double base = WQ[q] * h->p.rho0;
    switch (h->prec) {
      case 0: f[k] = ((const double*)raw.data())[k]; break;
      case 1: f[k] = ((const float*)raw.data())[k]; break;
      case 2: f[k] = (float)((float)base + half_to_float(((const uint16_t*)raw.data())[k]) * (float)inv); break;
      default: f[k] = (float)((float)base + bf16_to_float(((const uint16_t*)raw.data())[k]) * (float)inv); break;
    }
  }
  return SUSP_OK;
}

susp_status susp_set_populations(susp* h, const double* f) {
  if (!h || !f) return fail(SUSP_EINVAL, "NULL argument");
  const long long nc = h->v.ncell, tot = 19 * nc;
  const size_t es = esize(h->prec);
  std::vector<char> raw(tot * es);
  for (long long k = 0; k < tot; ++k) {
    const int q = (int)(k / nc);
    const double base = WQ[q] * h->p.rho0;
    switch (h->prec) {
      case 0: ((double*)raw.data())[k] = f[k]; break;
      case 1: ((float*)raw.data())[k] = (float)f[k]; break;
      case 2: ((uint16_t*)raw.data())[k] = float_to_half((float)((f[k] - base) * h->scale)); break;
      default: ((uint16_t*)raw.data())[k] = float_to_bf16((float)((f[k] - base) * h->scale)); break;
    }
  }
  susp_status st = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (st) return st;
  st = cuda_check(cudaMemcpy(h->fin, raw.data(), raw.size(), cudaMemcpyHostToDevice), "write populations");
  if (st) return st;
  refresh_links(h);
  return device_status(h);
}

susp_status susp_get_owner(susp* h, int32_t* owner) {
  if (!h || !owner) return fail(SUSP_EINVAL, "NULL argument");
  susp_status st = device_status(h);
  if (st) return st;
  return cuda_check(cudaMemcpy(owner, h->v.owner, 4 * h->v.ncell, cudaMemcpyDeviceToHost), "read owner");
}

susp_status susp_get_time(susp* h, int64_t* t, double* delta) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  susp_status st = device_status(h);
  if (st) return st;
  Proto pr;
  st = cuda_check(cudaMemcpy(&pr, h->v.proto, sizeof pr, cudaMemcpyDeviceToHost), "read protocol");
  if (st) return st;
  if (t) *t = pr.t;
  if (delta) *delta = pr.delta;
  return SUSP_OK;
}

susp_status susp_get_info(susp* h, susp_info* info) {
  if (!h || !info) return fail(SUSP_EINVAL, "NULL argument");
  const View& v = h->v;
  int dem = 0;
  if (v.move && v.n > 0) dem = v.nsub * ((v.brute ? 0 : 4) + 2);
  info->dem_substeps = v.nsub;
  info->launches_per_step = 2 + dem + 1 + (v.n > 0 ? 3 : 0);
  info->brute_force_pairs = v.brute;
  info->ncell = v.ncell;
  info->workspace_bytes = h->L.total;
  return SUSP_OK;
}

susp_status susp_profile(susp* h, int enable) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  if (enable && h->ev.empty()) {
    h->ev.resize(2 * PROF_MAX);
    for (auto& e : h->ev) {
      susp_status st = cuda_check(cudaEventCreate(&e), "cudaEventCreate");
      if (st) return st;
    }
  }
  h->prof = enable != 0;
  h->prof_n = 0;
  return SUSP_OK;
}

susp_status susp_profile_read(susp* h, double* ms_total, int* launches) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  susp_status st = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (st) return st;
  double tot = 0.0;
  for (int k = 0; k < h->prof_n; ++k) {
    float ms = 0.0f;
    st = cuda_check(cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]), "cudaEventElapsedTime");
    if (st) return st;
    tot += ms;
  }
  if (ms_total) *ms_total = tot;
  if (launches) *launches = h->prof_n;
  h->prof_n = 0;
  return SUSP_OK;
}

void susp_destroy(susp* h) {
  if (!h) return;
  for (auto& e : h->ev) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"
