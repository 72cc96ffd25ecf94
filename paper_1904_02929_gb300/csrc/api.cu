// api.cu — C ABI (include/susp.h): workspace layout, step sequencing, the
// per-step stress / protocol finalisation kernel and host-side read-back.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/susp.h"
#include "susp_dev.cuh"
#include "finalize.cuh"

using namespace susp_dev;

// launchers defined in the other translation units
void launch_plane_moments(int prec, const Batch& B, int total, cudaStream_t s);
void launch_collide_stream(int prec, const Batch& B, int grid, int staged, cudaStream_t s);
int lb_tensor_maps(int prec, int nx, int ny, int nz, void* fa, void* fb, void* owner, void* out);
int lb_blocks(int nx, int ny, int nz, int tile_lg, int staged);
void lb_occupancy(int prec, int staged, int* per_sm, int* sms);
void launch_claim(int prec, const Batch& B, int nparts, cudaStream_t s);
void launch_node_update(int prec, const Batch& B, int nparts, cudaStream_t s);
void launch_links(int prec, const Batch& B, int nparts, cudaStream_t s);
void launch_init_pop(int prec, const View& v, void* f, cudaStream_t s);
void launch_write_plb(const View& v, int plb_double, cudaStream_t s);
cudaError_t launch_dem_step(const Batch& B, int nparts, int ncells, int plb_double, int grid, cudaStream_t s);
int dem_grid_blocks(int plb_double, int n);

namespace {

thread_local std::string g_err = "";

susp_status fail(susp_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

const int HSLOTS = HSLOTS_DEV;   // tangential springs per particle (partners with larger index)
const double KPI = 3.14159265358979323846;

size_t esize(int prec) { return prec == 0 ? 8 : (prec == 1 ? 4 : 2); }
size_t csize(int prec) { return prec == 0 ? 8 : 4; }
size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Compensated time sums per box: 45 stress components (viscous, stresslet,
// contact and double-layer virials, lubrication stresslets, 3 x 3 each) and
// the two phase-weighted shear-stress sums of Eq. 17, 18; followed by as
// many compensation terms.

struct Layout {
  size_t fa, fb, owner, pm, pm2, vacc, views, tabs;
  size_t R, U, W, R2, U2, W2, pcx, rad, amap, mass, inert, imass, iinert, plb, Fh, Th, Fcov, Tcov, Fp, Tp;
  size_t Ro, m32a, m32b, pd, pk;
  size_t cstart, ccnt, cids, pcell, pj, ph, pcnt, pconst, drv;
  size_t hc0, hp0, hv0, hc1, hp1, hv1;
  size_t sums, hist, counters, proto, err, tmap, plbn, res;
  size_t total;
  int ncx, ncy, ncz, brute, ncells;
  double csx, csy, csz, hrange;
};

bool valid(const susp_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return false; }
  if (p->nx < 4 || p->ny < 4 || p->nz < 4) { why = "lattice dims must be >= 4"; return false; }
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 27)) { why = "lattice larger than 2^27 nodes"; return false; }
  if (p->nx > 2047 || p->ny > 2047 || p->nz > 1023) { why = "lattice dims must be <= 2047 x 2047 x 1023"; return false; }
  if (!(p->tau > 0.5)) { why = "tau must exceed 1/2"; return false; }
  if (p->collision != 0 && p->collision != 1) { why = "collision must be 0 (BGK) or 1 (Ladd)"; return false; }
  if (p->collision == 1 && p->tau_bulk > 0.0 && !(p->tau_bulk > 0.5)) { why = "tau_bulk must exceed 1/2"; return false; }
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
      for (int c = 0; c < 3; ++c)
        if (!std::isfinite(p->pos[3 * i + c])) { why = "particle centres must be finite"; return false; }
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

// The block of susp_read_results: the error word (padded to 8 bytes), the
// two sample counters, the NSUMS stress sums, the 3 nbins histogram, then
// the centres, velocities and spins (3 n doubles each).
static size_t results_bytes(int n, int nbins) {
  return 8 + 16 + 8 * (size_t)NSUMS + 24 * (size_t)nbins + 72 * (size_t)n;
}
static const size_t RES_CNT = 8, RES_SUMS = 24;
static size_t res_hist() { return RES_SUMS + 8 * (size_t)NSUMS; }
static size_t res_parts(int nbins) { return res_hist() + 24 * (size_t)nbins; }

void make_layout(const susp_params* p, Layout& L) {
  const long long nc = (long long)p->nx * p->ny * p->nz;
  const int n = p->n, nn = n > 0 ? n : 1;
  const int prec = p->prec;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
  L.fa = take(19 * nc * esize(prec));
  L.fb = take(19 * nc * esize(prec));
  L.owner = take(4 * nc);
  L.pm = take(2ULL * p->nx * p->nz * 4 * csize(prec));
  L.pm2 = take(2ULL * p->nx * p->nz * 4 * csize(prec));
  L.vacc = take(ACC_REP * ACC_STRIDE * 8);
  L.views = take(sizeof(View));
  L.tabs = take(4 * 2 * sizeof(int));   // the one-box batch tables
  L.R = take(24 * nn); L.U = take(24 * nn); L.W = take(24 * nn);
  L.R2 = take(24 * nn); L.U2 = take(24 * nn); L.W2 = take(24 * nn); L.pcx = take(4 * 8 * (size_t)nn);
  L.Ro = take(24 * nn); L.m32a = take(48 * nn); L.m32b = take(48 * nn);
  L.rad = take(8 * nn); L.amap = take(8 * nn); L.mass = take(8 * nn); L.inert = take(8 * nn);
  L.imass = take(8 * nn); L.iinert = take(8 * nn);
  L.plb = take(12 * csize(prec) * nn);
  L.Fh = take(24 * nn); L.Th = take(24 * nn); L.Fcov = take(24 * nn); L.Tcov = take(24 * nn);
  L.Fp = take(24 * nn); L.Tp = take(24 * nn);
  // cell list geometry
  double amax = 0.0;
  for (int i = 0; i < n; ++i) amax = std::max(amax, p->radius[i]);
  L.hrange = hrange_of(p);
  const double cmin = 2.0 * amax + L.hrange + 1.0;
  int ncx = (int)floor(p->nx / cmin), ncy = (int)floor(p->ny / cmin), ncz = (int)floor(p->nz / cmin);
  // up to BRUTE_PAIRS_MAX particles every warp scans all particles for its
  // candidates (cheaper than building the cell list); beyond, the cell list
  if (ncx < 3 || ncy < 3 || n <= BRUTE_PAIRS_MAX) { ncx = ncy = ncz = 1; L.brute = 1; }
  else { L.brute = 0; if (ncz < 1) ncz = 1; }
  L.ncx = ncx; L.ncy = ncy; L.ncz = ncz;
  L.ncells = ncx * ncy * ncz;
  L.csx = (double)p->nx / ncx; L.csy = (double)p->ny / ncy; L.csz = (double)p->nz / ncz;
  L.pj = take(4 * (size_t)nn * PAIR_SLOTS); L.ph = take(24 * (size_t)nn * PAIR_SLOTS); L.pcnt = take(4 * nn); L.pconst = take(64 * (size_t)nn); L.drv = take(4 * (size_t)nn);
  L.pd = take(16 * (size_t)nn * PAIR_SLOTS); L.pk = take((size_t)nn * PAIR_SLOTS);
  L.cstart = take(4 * (L.ncells + 1)); L.ccnt = take(4 * L.ncells);
  L.cids = take(4 * nn); L.pcell = take(4 * nn);
  L.hc0 = take(4 * nn); L.hp0 = take(4 * (size_t)nn * HSLOTS); L.hv0 = take(24 * (size_t)nn * HSLOTS);
  L.hc1 = take(4 * nn); L.hp1 = take(4 * (size_t)nn * HSLOTS); L.hv1 = take(24 * (size_t)nn * HSLOTS);
  L.sums = take(8 * 2 * NSUMS);
  int nb = p->nbins > 0 ? p->nbins : 36;
  L.hist = take(8 * 3 * nb);
  L.counters = take(8 * 4);
  L.proto = take(sizeof(Proto));
  L.err = take(4);
  L.tmap = take(384);   // three 128-byte tensor maps (256-byte aligned, as they must be 64)
  L.plbn = take(12 * csize(prec) * nn);   // the next step's copy (overlapped step)
  L.res = take(results_bytes(n, nb));     // staging block of susp_read_results
  L.total = o;
}

// ------------------------------------------------------------ device kernels

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

// End of step t, one block per box (boxes whose particles do not move;
// the particle kernel does the same after its last sub-step otherwise).
// End of the lattice step of box blockIdx.x.  plb16 > 0 (the overlapped
// step): first the particle kernel's copy of the next step, plb16 16-byte
// words per particle, goes into the copy that the node-map and link kernels
// read (boxes with moving particles only).
__global__ void __launch_bounds__(64) k_finalize(Batch B, int plb16) {
  const View& v = B.views[blockIdx.x];
  if (plb16 > 0 && v.move) {
    const float4* src = static_cast<const float4*>(v.plb_next);
    float4* dst = static_cast<float4*>(v.plb);
    for (int k = threadIdx.x; k < plb16 * v.n; k += blockDim.x) dst[k] = src[k];
  }
  finalize_box(v);
}

// The results block of one box (see results_bytes), gathered in 8-byte words.
__global__ void k_gather_results(View v, unsigned long long* __restrict__ dst) {
  const long long nsw = NSUMS, nhw = 3LL * v.nbins, npw = 3LL * v.n;
  const long long total = 3 + nsw + nhw + 3 * npw;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    unsigned long long w;
    if (k == 0) w = (unsigned long long)(unsigned)*v.err;
    else if (k < 3) w = v.counters[k - 1];
    else if (k < 3 + nsw) w = __double_as_longlong(v.sums[k - 3]);
    else if (k < 3 + nsw + nhw) w = __double_as_longlong(v.hist[k - 3 - nsw]);
    else {
      const long long j = k - 3 - nsw - nhw;
      const double* src = j < npw ? v.R : (j < 2 * npw ? v.U : v.W);
      w = __double_as_longlong(src[j % npw]);
    }
    dst[k] = w;
  }
}

// Error words of the boxes of a batch, in batch order.
__global__ void k_gather_err(Batch B, int* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B.nbox) out[b] = *B.views[b].err;
}

}  // namespace

// ------------------------------------------------------------ step engine

struct GraphSlot {
  bool valid = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t nodes[6] = {};   // event-record nodes at the stage boundaries (profiled graph)
};

static const int PROF_MAX = 4096;

// The launch sequence of one lattice step over a set of boxes (a single box,
// or the boxes attached to a batch).  Every kernel takes the whole set; the
// population buffers and spring tables of each box follow from its own step
// counter on the device, so one captured graph serves every step.
struct Engine {
  int prec = 0;
  Batch B{};                 // device views and prefix tables
  int nbox = 0, nparts = 0, ncells = 0, nplane = 0, ntiles = 0;
  bool any_move = false;     // some box has moving particles
  int lb_grid = 1, dem_grid = 1;
  int tile_lg = 3;           // collide-stream tile height 2^tile_lg (the tuner's choice)
  int bps = 0;               // its resident blocks per SM (0: as many as fit)
  int staged = 0;            // source rows staged by tensor copies (128 x 4 tiles, tile_lg 2)
  // The collide-stream beside the particle kernel: asked for (overlap), and
  // in effect (ov_active) when the particles move, the collide grid has one
  // block per SM and the particle grid fits one block per SM beside it.  It
  // runs on the side stream, forked from and joined to the engine's stream.
  int overlap = 0;
  bool ov_active = false;
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaStream_t stream = nullptr;
  bool use_graphs = true;
  GraphSlot graphs[2];       // [timed]
  bool prof = false;
  int prof_n = 0;
  std::vector<cudaEvent_t> ev;
};

static susp_status cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(SUSP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return SUSP_OK;
}

// Host copy of the prefix tables for the views of a set of boxes; fills the
// engine's totals.  tabs receives tile, particle, plane, cell tables of
// nbox + 1 entries each.
static void eng_tables(Engine& e, const std::vector<const View*>& vs, std::vector<int>& tabs) {
  const int nb = (int)vs.size();
  tabs.assign(4 * (nb + 1), 0);
  int* tile = tabs.data();
  int* part = tile + (nb + 1);
  int* plane = part + (nb + 1);
  int* cell = plane + (nb + 1);
  e.any_move = false;
  int msub = 1;
  for (int b = 0; b < nb; ++b) {
    const View& v = *vs[b];
    tile[b + 1] = tile[b] + lb_blocks(v.nx, v.ny, v.nz, e.tile_lg, e.staged && e.prec >= 1);
    part[b + 1] = part[b] + v.n;
    plane[b + 1] = plane[b] + 2 * v.nx * v.nz;
    cell[b + 1] = cell[b] + (v.brute ? 0 : v.ncells);
    if (v.move && v.n > 0) { e.any_move = true; msub = std::max(msub, v.nsub); }
  }
  e.nbox = nb;
  e.ntiles = tile[nb]; e.nparts = part[nb]; e.nplane = plane[nb]; e.ncells = cell[nb];
  e.B.nbox = nb;
  e.B.max_nsub = msub;
  e.B.tile_lg = e.tile_lg;
  int per = 1, sms = 1;
  lb_occupancy(e.prec, e.staged, &per, &sms);
  const int bps = (e.bps >= 1 && e.bps <= per) ? e.bps : per;
  e.lb_grid = std::max(1, std::min(sms * bps, e.ntiles));
  e.dem_grid = dem_grid_blocks(e.prec == 0, e.nparts);
  e.ov_active = e.overlap && e.side && e.any_move && e.nparts > 0 && bps == 1 && e.dem_grid <= sms;
  e.B.dem_fin = e.ov_active ? 0 : 1;
}

// The side stream and fork / join events of the overlapped step.
static susp_status eng_side(Engine& e) {
  if (e.side) return SUSP_OK;
  susp_status st = cuda_check(cudaStreamCreateWithFlags(&e.side, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!st) st = cuda_check(cudaEventCreateWithFlags(&e.fork_ev, cudaEventDisableTiming), "cudaEventCreate");
  if (!st) st = cuda_check(cudaEventCreateWithFlags(&e.join_ev, cudaEventDisableTiming), "cudaEventCreate");
  return st;
}

// Point the engine's batch at device storage for nbox views and the tables.
static void eng_bind(Engine& e, char* views, char* tabs, int nbox) {
  e.B.views = (const View*)views;
  const int* t = (const int*)tabs;
  e.B.tile_off = t;
  e.B.part_off = t + (nbox + 1);
  e.B.plane_off = t + 2 * (nbox + 1);
  e.B.cell_off = t + 3 * (nbox + 1);
}

static void eng_drop_graphs(Engine& e) {
  for (auto& g : e.graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = GraphSlot();
  }
}

// Stage boundaries recorded when a step is profiled: start, after the
// collide-stream (which also writes the next step's Lees-Edwards plane
// moments), the particle sub-steps (cell list included), the finalisation,
// the node-map update, and the boundary links.
static const int NEV = 6;

// The launches of one lattice step; evs (optional, NEV events) mark the stage
// boundaries.
static cudaError_t eng_enqueue(Engine& e, const cudaEvent_t* evs) {
  cudaStream_t s = e.stream;
  cudaError_t err = cudaSuccess;
  const bool dem = e.any_move && e.nparts > 0;
  if (evs) cudaEventRecord(evs[0], s);
  if (e.ov_active) {
    // Within a step the collide-stream needs neither the particle sub-steps
    // nor their results (it reads the particle copy of step t, which they do
    // not write), so it runs on the side stream beside them; the
    // finalisation waits for both.  Stage times: the collide-stream, then
    // the particle time not hidden behind it.
    cudaEventRecord(e.fork_ev, s);
    cudaStreamWaitEvent(e.side, e.fork_ev, 0);
    launch_collide_stream(e.prec, e.B, e.lb_grid, e.staged, e.side);
    if (evs) cudaEventRecord(evs[1], e.side);
    cudaEventRecord(e.join_ev, e.side);
    err = launch_dem_step(e.B, e.nparts, e.ncells, e.prec == 0, e.dem_grid, s);
    cudaStreamWaitEvent(s, e.join_ev, 0);
    if (evs) cudaEventRecord(evs[2], s);
    k_finalize<<<e.nbox, 64, 0, s>>>(e.B, (int)(12 * csize(e.prec) / 16));
    if (evs) cudaEventRecord(evs[3], s);
  } else {
    launch_collide_stream(e.prec, e.B, e.lb_grid, e.staged, s);
    if (evs) cudaEventRecord(evs[1], s);
    // the particle kernel ends with the finalisation when it runs
    if (dem) err = launch_dem_step(e.B, e.nparts, e.ncells, e.prec == 0, e.dem_grid, s);
    if (evs) cudaEventRecord(evs[2], s);
    if (!dem) k_finalize<<<e.nbox, 64, 0, s>>>(e.B, 0);
    if (evs) cudaEventRecord(evs[3], s);
  }
  launch_node_update(e.prec, e.B, e.nparts, s);
  if (evs) cudaEventRecord(evs[4], s);
  launch_links(e.prec, e.B, e.nparts, s);
  if (evs) cudaEventRecord(evs[5], s);
  return err != cudaSuccess ? err : cudaGetLastError();
}

// Capture one step as a CUDA graph (timed: with event-record nodes that each
// replay retargets); false if capture is not possible on this stream.
static bool eng_capture(Engine& e, int timed) {
  GraphSlot& g = e.graphs[timed];
  cudaStream_t s = e.stream;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaError_t le = eng_enqueue(e, timed ? e.ev.data() : nullptr);
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (le != cudaSuccess || ce != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return false;
  }
  for (auto& n : g.nodes) n = nullptr;
  if (timed) {
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev = nullptr;
      cudaGraphEventRecordNodeGetEvent(nd, &ev);
      for (int k = 0; k < NEV; ++k)
        if (ev == e.ev[k]) g.nodes[k] = nd;
    }
    for (int k = 0; k < NEV; ++k)
      if (!g.nodes[k]) {
        cudaGraphDestroy(graph);
        return false;
      }
  }
  if (cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  g.graph = graph;
  g.valid = true;
  return true;
}

static susp_status eng_step(Engine& e, int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    const int timed = (e.prof && e.prof_n < PROF_MAX) ? 1 : 0;
    const cudaEvent_t* evs = timed ? e.ev.data() + (size_t)NEV * e.prof_n : nullptr;
    bool done = false;
    if (e.use_graphs && e.stream != nullptr) {
      if (!e.graphs[timed].valid && !eng_capture(e, timed)) e.use_graphs = false;
      if (e.use_graphs) {
        GraphSlot& g = e.graphs[timed];
        if (timed)
          for (int k = 0; k < NEV; ++k) cudaGraphExecEventRecordNodeSetEvent(g.exec, g.nodes[k], evs[k]);
        done = cudaGraphLaunch(g.exec, e.stream) == cudaSuccess;
        if (!done) { cudaGetLastError(); e.use_graphs = false; }
      }
    }
    if (!done) {
      susp_status st = cuda_check(eng_enqueue(e, evs), "step launch");
      if (st) return st;
    }
    if (timed) ++e.prof_n;
  }
  return cuda_check(cudaGetLastError(), "launch");
}

static susp_status eng_profile(Engine& e, int enable) {
  if (enable && e.ev.empty()) {
    e.ev.resize((size_t)NEV * PROF_MAX);
    for (auto& x : e.ev) {
      susp_status st = cuda_check(cudaEventCreate(&x), "cudaEventCreate");
      if (st) return st;
    }
  }
  e.prof = enable != 0;
  e.prof_n = 0;
  return SUSP_OK;
}

// Summed stage times of the profiled steps (ms[NEV - 1]); starts a new window.
static susp_status eng_profile_stages(Engine& e, double* ms, int* steps) {
  susp_status st = cuda_check(cudaStreamSynchronize(e.stream), "sync");
  if (st) return st;
  double tot[NEV - 1] = {0, 0, 0, 0, 0};
  for (int k = 0; k < e.prof_n; ++k)
    for (int j = 0; j + 1 < NEV; ++j) {
      float m = 0.0f;
      st = cuda_check(cudaEventElapsedTime(&m, e.ev[(size_t)NEV * k + j], e.ev[(size_t)NEV * k + j + 1]),
                      "cudaEventElapsedTime");
      if (st) return st;
      tot[j] += m;
    }
  if (ms)
    for (int j = 0; j + 1 < NEV; ++j) ms[j] = tot[j];
  if (steps) *steps = e.prof_n;
  e.prof_n = 0;
  return SUSP_OK;
}

static susp_status eng_profile_read(Engine& e, double* ms_total, int* launches) {
  double ms[NEV - 1];
  susp_status st = eng_profile_stages(e, ms, launches);
  if (st) return st;
  if (ms_total) *ms_total = ms[0];
  return SUSP_OK;
}

static void eng_release(Engine& e) {
  if (e.stream) cudaStreamSynchronize(e.stream);
  if (e.side) cudaStreamSynchronize(e.side);
  eng_drop_graphs(e);
  for (auto& x : e.ev) cudaEventDestroy(x);
  e.ev.clear();
  if (e.fork_ev) cudaEventDestroy(e.fork_ev);
  if (e.join_ev) cudaEventDestroy(e.join_ev);
  if (e.side) cudaStreamDestroy(e.side);
  e.fork_ev = e.join_ev = nullptr;
  e.side = nullptr;
}

// Clear the viscous-stress sums of the current step of every box.
__global__ void k_zero_visc(Batch B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B.nbox)
    for (int r = 0; r < ACC_REP; ++r)
      for (int k = 0; k < 6; ++k) B.views[b].step_acc[r * ACC_STRIDE + k] = 0.0;
}

// Launch-shape tuner: times the collide-stream over the set's own boxes for
// tile heights of 4, 8 and 16 rows and each count of resident blocks per SM
// the occupancy allows, and keeps the fastest.  At a step boundary the
// collide-stream is a pure function of the buffer it reads and overwrites
// the other one, which the next step rewrites, so the trial launches leave
// the state alone but for the viscous-stress sums, cleared afterwards (they
// are zero at a step boundary).  tabs_dev: the device copy of the prefix
// tables, rewritten for each trial shape.  Synchronises.
static susp_status eng_tune(Engine& e, const std::vector<const View*>& vs, char* tabs_dev, int* tile_rows,
                            int* blocks_per_sm, double* us) {
  cudaStream_t s = e.stream;
  susp_status st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (st) return st;
  eng_drop_graphs(e);
  // candidate shapes: the direct kernel at tile heights 4, 8, 16 and the
  // staged one (128 x 4 tiles; FP32 / FP16 / BF16 boxes with tensor maps),
  // each at every resident block count the occupancy allows
  bool any_map = false;
  for (const View* v : vs) any_map = any_map || v->tmap != nullptr;
  cudaEvent_t ea = nullptr, eb = nullptr;
  st = cuda_check(cudaEventCreate(&ea), "cudaEventCreate");
  if (!st) st = cuda_check(cudaEventCreate(&eb), "cudaEventCreate");
  const int reps = 3;
  double best = 1e300;
  int best_lg = e.tile_lg, best_bps = e.bps, best_staged = e.staged;
  std::vector<int> tabs;
  for (int staged = 0; staged <= ((e.prec >= 1 && any_map) ? 1 : 0) && !st; ++staged) {
    int per = 1, sms = 1;
    lb_occupancy(e.prec, staged, &per, &sms);
    for (int lg = 2; lg <= (staged ? 2 : 4) && !st; ++lg)
      for (int bps = 1; bps <= per && !st; ++bps) {
        e.tile_lg = lg;
        e.bps = bps;
        e.staged = staged;
        eng_tables(e, vs, tabs);
        cudaMemcpyAsync(tabs_dev, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, s);
        launch_plane_moments(e.prec, e.B, e.nplane, s);
        launch_collide_stream(e.prec, e.B, e.lb_grid, e.staged, s);   // warm-up
        cudaEventRecord(ea, s);
        for (int r = 0; r < reps; ++r) launch_collide_stream(e.prec, e.B, e.lb_grid, e.staged, s);
        cudaEventRecord(eb, s);
        st = cuda_check(cudaEventSynchronize(eb), "tuning launch");
        float ms = 0.0f;
        if (!st) st = cuda_check(cudaEventElapsedTime(&ms, ea, eb), "cudaEventElapsedTime");
        if (!st && ms / reps < best) { best = ms / reps; best_lg = lg; best_bps = bps; best_staged = staged; }
      }
  }
  if (ea) cudaEventDestroy(ea);
  if (eb) cudaEventDestroy(eb);
  // The fastest shape, with the step in sequence: the overlapped step is
  // only taken on request (susp_set_overlap).  On the 96^3 suspension the
  // collide-stream beside the particle kernel took 127 us against 47 us
  // alone and the step 0.232 ms against 0.193 ms: the two kernels slow each
  // other down far more than the overlap hides.
  e.tile_lg = best_lg;
  e.bps = best_bps;
  e.staged = best_staged;
  e.overlap = 0;
  eng_tables(e, vs, tabs);
  cudaMemcpyAsync(tabs_dev, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, s);
  k_zero_visc<<<(e.nbox + 127) / 128, 128, 0, s>>>(e.B);
  susp_status st2 = cuda_check(cudaStreamSynchronize(s), "tuner");
  if (st) return st;
  if (st2) return st2;
  int per = 1, sms = 1;
  lb_occupancy(e.prec, e.staged, &per, &sms);
  if (tile_rows) *tile_rows = 1 << e.tile_lg;
  if (blocks_per_sm) *blocks_per_sm = std::max(1, std::min(e.bps, per));
  if (us) *us = 1e3 * best;
  return SUSP_OK;
}

// Set the collide-stream launch shape explicitly (the tuner's alternative).
static susp_status eng_set_shape(Engine& e, const std::vector<const View*>& vs, char* tabs_dev, int tile_rows,
                                 int blocks_per_sm, int staged) {
  int lg = tile_rows == 4 ? 2 : tile_rows == 8 ? 3 : tile_rows == 16 ? 4 : -1;
  if (lg < 0) return fail(SUSP_EINVAL, "tile_rows must be 4, 8 or 16");
  if (staged != 0 && staged != 1) return fail(SUSP_EINVAL, "staged must be 0 or 1");
  if (staged && (e.prec < 1 || lg != 2))
    return fail(SUSP_EINVAL, "the staged collide-stream needs FP32 / FP16 / BF16 storage and tile_rows = 4");
  if (blocks_per_sm < 1) return fail(SUSP_EINVAL, "blocks_per_sm must be >= 1");
  cudaStream_t s = e.stream;
  susp_status st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (st) return st;
  eng_drop_graphs(e);
  e.tile_lg = lg;
  e.bps = blocks_per_sm;
  e.staged = staged;
  std::vector<int> tabs;
  eng_tables(e, vs, tabs);
  cudaMemcpyAsync(tabs_dev, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, s);
  return cuda_check(cudaStreamSynchronize(s), "set launch shape");
}

static susp_status eng_set_overlap(Engine& e, const std::vector<const View*>& vs, char* tabs_dev, int enable) {
  if (enable != 0 && enable != 1) return fail(SUSP_EINVAL, "enable must be 0 or 1");
  cudaStream_t s = e.stream;
  susp_status st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (st) return st;
  if (enable) {
    st = eng_side(e);
    if (st) return st;
    e.bps = 1;
  }
  eng_drop_graphs(e);
  e.overlap = enable;
  std::vector<int> tabs;
  eng_tables(e, vs, tabs);
  cudaMemcpyAsync(tabs_dev, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, s);
  return cuda_check(cudaStreamSynchronize(s), "set overlap");
}

static void eng_get_shape(const Engine& e, int* tile_rows, int* blocks_per_sm, int* staged) {
  int per = 1, sms = 1;
  lb_occupancy(e.prec, e.staged, &per, &sms);
  if (tile_rows) *tile_rows = 1 << e.tile_lg;
  if (blocks_per_sm) *blocks_per_sm = (e.bps >= 1 && e.bps <= per) ? e.bps : per;
  if (staged) *staged = e.staged;
}

// ------------------------------------------------------------ handles

struct susp {
  susp_params p;
  int prec;
  Layout L;
  View v;
  char* ws;
  bool have_shear;
  susp_shear shear;
  std::vector<double> radius;
  double scale;
  Engine eng;                 // the box stepped alone (a batch of one)
  susp_batch* batch;          // batch the box is attached to, or NULL
  std::vector<unsigned char> maps;   // host copy of the tensor maps (device addresses of this workspace)
};

struct susp_batch {
  int max_boxes;
  int prec;
  char* ws;
  Engine eng;
  std::vector<susp*> boxes;
};

static cudaStream_t stream_of(const susp* h) { return h->batch ? h->batch->eng.stream : h->eng.stream; }

// Status for a box's device error word.
static susp_status err_status(int err) {
  if (err & ERR_OVERLAP) return fail(SUSP_EOVERLAP, "two mapped spheres claimed one node");
  if (err & ERR_UNSTABLE) return fail(SUSP_EUNSTABLE, "non-positive density or particle speed >= 0.5");
  if (err & ERR_LINKS) return fail(SUSP_ENOMEM, "particle surface larger than the link kernel stages");
  if (err & ERR_PAIRS) return fail(SUSP_ENOMEM, "tangential-spring table full");
  if (err & ERR_TIMEOUT) return fail(SUSP_ETIMEOUT, "a bounded device wait gave up");
  return SUSP_OK;
}

static susp_status device_status(susp* h) {
  cudaError_t e = cudaStreamSynchronize(stream_of(h));
  if (e != cudaSuccess) return fail(SUSP_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
  int err = 0;
  e = cudaMemcpy(&err, h->v.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(SUSP_ECUDA, std::string("read error flag: ") + cudaGetErrorString(e));
  return err_status(err);
}

// Rebuild the boundary links of this box from its current populations (the
// stresslet sum they feed to the next finalisation starts again from zero).
static void refresh_links(susp* h) {
  for (int r = 0; r < ACC_REP; ++r)
    cudaMemsetAsync(h->v.step_acc + r * ACC_STRIDE + 6, 0, 9 * sizeof(double), stream_of(h));
  launch_links(h->prec, h->eng.B, h->v.n, stream_of(h));
}

static Proto read_proto(susp* h) {
  Proto pr;
  cudaMemcpy(&pr, h->v.proto, sizeof pr, cudaMemcpyDeviceToHost);
  return pr;
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
  h->have_shear = false;
  h->batch = nullptr;
  h->radius.assign(p->radius, p->radius + p->n);
  h->scale = p->prec == SUSP_FP16_DEV ? 4096.0 : 1.0;
  char* w = h->ws;
  View& v = h->v;
  memset(&v, 0, sizeof(View));
  const int n = p->n;
  v.nx = p->nx; v.ny = p->ny; v.nz = p->nz;
  v.ncell = (long long)p->nx * p->ny * p->nz;
  v.tau = p->tau; v.rho0 = p->rho0;
  for (int a = 0; a < 3; ++a) { v.g[a] = p->body_force[a]; v.g_f[a] = (float)p->body_force[a]; }
  v.has_g = (p->body_force[0] != 0.0 || p->body_force[1] != 0.0 || p->body_force[2] != 0.0);
  v.scale = (float)h->scale; v.inv_scale = (float)(1.0 / h->scale);
  v.omega_d = 1.0 / p->tau; v.vf_d = -(1.0 - 0.5 / p->tau);
  v.omega_f = (float)v.omega_d; v.vf_f = (float)v.vf_d; v.rho0_f = (float)p->rho0;
  {
    const double taub = p->tau_bulk > 0.0 ? p->tau_bulk : p->tau;
    v.ladd = p->collision == 1;
    v.ls_d = 1.0 - 1.0 / p->tau; v.lb_d = 1.0 - 1.0 / taub; v.vfb_d = -(1.0 - 0.5 / taub);
    v.ls_f = (float)v.ls_d; v.lb_f = (float)v.lb_d; v.vfb_f = (float)v.vfb_d;
  }
  v.inv_nx_d = 1.0 / p->nx; v.inv_ny_d = 1.0 / p->ny; v.inv_nz_d = 1.0 / p->nz;
  v.inv_nx_f = (float)v.inv_nx_d; v.inv_ny_f = (float)v.inv_ny_d; v.inv_nz_f = (float)v.inv_nz_d;
  v.fa = w + L.fa; v.fb = w + L.fb;
  v.step_acc = (double*)(w + L.vacc);
  v.owner = (int*)(w + L.owner);
  v.plane_mom = w + L.pm;
  v.plane_mom2 = w + L.pm2;
  v.n = n;
  v.R = (double*)(w + L.R); v.U = (double*)(w + L.U); v.W = (double*)(w + L.W);
  v.R2 = (double*)(w + L.R2); v.U2 = (double*)(w + L.U2); v.W2 = (double*)(w + L.W2);
  v.Ro = (double*)(w + L.Ro); v.m32[0] = (float*)(w + L.m32a); v.m32[1] = (float*)(w + L.m32b);
  v.pd = (float4*)(w + L.pd); v.pk = (signed char*)(w + L.pk);
  v.pcx = (int*)(w + L.pcx);
  v.rad = (double*)(w + L.rad); v.amap = (double*)(w + L.amap);
  v.mass = (double*)(w + L.mass); v.inert = (double*)(w + L.inert);
  v.inv_m = (double*)(w + L.imass); v.inv_I = (double*)(w + L.iinert);
  v.plb = w + L.plb;
  v.plb_next = w + L.plbn;
  v.Fh = (double*)(w + L.Fh); v.Th = (double*)(w + L.Th);
  v.Fcov = (double*)(w + L.Fcov); v.Tcov = (double*)(w + L.Tcov);
  v.Fp = (double*)(w + L.Fp); v.Tp = (double*)(w + L.Tp);
  v.ncx = L.ncx; v.ncy = L.ncy; v.ncz = L.ncz; v.brute = L.brute; v.ncells = L.ncells;
  v.csx = L.csx; v.csy = L.csy; v.csz = L.csz;
  v.inv_csx = 1.0 / L.csx; v.inv_csy = 1.0 / L.csy; v.inv_csz = 1.0 / L.csz;
  v.cell_start = (int*)(w + L.cstart); v.cell_cnt = (int*)(w + L.ccnt);
  v.cell_ids = (int*)(w + L.cids); v.pcell = (int*)(w + L.pcell);
  v.pj = (int*)(w + L.pj); v.ph = (double*)(w + L.ph); v.pcnt = (int*)(w + L.pcnt); v.pconst = (void*)(w + L.pconst); v.drv = (int*)(w + L.drv);
  v.has_drv = 0;
  for (int i = 0; p->driven && i < n; ++i) v.has_drv |= p->driven[i] != 0;
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
  v.dt_sub = 1.0 / v.nsub;
  {
    PairConst<double>& d = v.pc_d;
    d.kn = v.kn; d.kt = v.kt; d.eta_n = v.eta_n; d.mu = v.mu; d.F0 = v.F0; d.debye = v.debye;
    d.debye10 = 10.0 * v.debye; d.lub_cut = v.lub_cut; d.lub_delta = v.lub_delta; d.eta0 = v.eta0;
    d.hrange = v.hrange; d.rep = v.F0 > 0.0; d.lub = v.lub_cut > 0.0;
    PairConst<float>& f = v.pc_f;
    f.kn = (float)d.kn; f.kt = (float)d.kt; f.eta_n = (float)d.eta_n; f.mu = (float)d.mu;
    f.F0 = (float)d.F0; f.debye = (float)d.debye; f.debye10 = (float)d.debye10;
    f.lub_cut = (float)d.lub_cut; f.lub_delta = (float)d.lub_delta; f.eta0 = (float)d.eta0;
    f.hrange = (float)d.hrange; f.rep = d.rep; f.lub = d.lub;
  }
  v.sums = (double*)(w + L.sums); v.hist = (double*)(w + L.hist);
  v.counters = (unsigned long long*)(w + L.counters);
  v.proto = (Proto*)(w + L.proto); v.err = (int*)(w + L.err);
  std::vector<unsigned char>& maps = h->maps;
  maps.assign(384, 0);
  v.tmap = lb_tensor_maps(h->prec, v.nx, v.ny, v.nz, v.fa, v.fb, v.owner, maps.data()) ? (const void*)(w + L.tmap)
                                                                                    : nullptr;

  Engine& e = h->eng;
  e.prec = h->prec;
  e.stream = (cudaStream_t)cuda_stream;
  std::vector<int> tabs;
  eng_tables(e, std::vector<const View*>{&v}, tabs);
  eng_bind(e, w + L.views, w + L.tabs, 1);

  cudaStream_t s = e.stream;
  susp_status st = SUSP_OK;
  // zero everything past the populations, then fill
  st = cuda_check(cudaMemsetAsync(w + L.owner, 0, L.total - L.owner, s), "memset workspace");
  if (st) { eng_release(h->eng); delete h; return st; }
  cudaMemsetAsync(v.owner, 0xff, 4 * v.ncell, s);
  if (v.tmap) cudaMemcpyAsync(w + L.tmap, maps.data(), 384, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(w + L.views, &v, sizeof(View), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(w + L.tabs, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, s);
  std::vector<double> zeros(3 * n, 0.0), im(n), iI(n);
  // centres into the box (the offset is zero at creation: plain periodic wrap)
  std::vector<double> R(p->pos, p->pos + 3 * n);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) {
      const double L = c == 0 ? p->nx : (c == 1 ? p->ny : p->nz);
      double& x = R[3 * i + c];
      x -= L * floor(x / L);
      if (!(x >= 0.0 && x < L)) x = 0.0;
    }
  if (n > 0) {
    for (int i = 0; i < n; ++i) {
      im[i] = 1.0 / mass[i];
      iI[i] = 1.0 / inert[i];
    }
    cudaMemcpyAsync(v.R, R.data(), 24 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.U, p->vel ? p->vel : zeros.data(), 24 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.W, p->omega ? p->omega : zeros.data(), 24 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.rad, p->radius, 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.amap, amap.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.mass, mass.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.inert, inert.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.inv_m, im.data(), 8 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.inv_I, iI.data(), 8 * n, cudaMemcpyHostToDevice, s);
  }
  std::vector<int> drv(n > 0 ? n : 1, 0);
  if (n > 0 && p->driven) {
    for (int i = 0; i < n; ++i) drv[i] = p->driven[i] != 0;
    cudaMemcpyAsync(v.drv, drv.data(), 4 * n, cudaMemcpyHostToDevice, s);
  }
  Proto pr;
  memset(&pr, 0, sizeof pr);
  pr.ny = p->ny;
  cudaMemcpyAsync(v.proto, &pr, sizeof pr, cudaMemcpyHostToDevice, s);
  // the copies above read pageable host memory: wait before it goes away
  st = cuda_check(cudaStreamSynchronize(s), "upload");
  if (st) { eng_release(h->eng); delete h; return st; }
  k_proto_set<<<1, 1, 0, s>>>(v.proto, v.nx, 0, 0.0, 0.0, 0.0, 0.0);
  launch_init_pop(h->prec, v, v.fa, s);
  launch_init_pop(h->prec, v, v.fb, s);
  launch_write_plb(v, h->prec == 0, s);
  launch_claim(h->prec, e.B, n, s);
  refresh_links(h);
  launch_plane_moments(h->prec, e.B, e.nplane, s);
  st = cuda_check(cudaGetLastError(), "launch");
  if (st) { eng_release(h->eng); delete h; return st; }
  st = device_status(h);
  if (st) { eng_release(h->eng); delete h; return st; }
  *out = h;
  return SUSP_OK;
}

// Set the box's shear protocol at its current step (no-op when unchanged).
static void set_shear(susp* h, const susp_shear* sh) {
  if (h->have_shear && memcmp(&h->shear, sh, sizeof(susp_shear)) == 0) return;
  k_proto_set<<<1, 1, 0, stream_of(h)>>>(h->v.proto, h->v.nx, sh->kind, sh->rate, sh->gamma0, sh->omega,
                                         sh->theta);
  refresh_links(h);   // the image velocity of the boundary links changed
  h->shear = *sh;
  h->have_shear = true;
}

susp_status susp_step(susp* h, int nsteps, const susp_shear* sh) {
  if (!h || !sh || nsteps < 0) return fail(SUSP_EINVAL, "bad argument to susp_step");
  if (sh->kind != 0 && sh->kind != 1) return fail(SUSP_EINVAL, "shear kind must be 0 or 1");
  if (h->batch && nsteps > 0) return fail(SUSP_ESTATE, "box is attached to a batch: step the batch");
  set_shear(h, sh);
  return eng_step(h->eng, nsteps);
}

susp_status susp_stress_reset(susp* h) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  cudaStream_t s = stream_of(h);
  cudaMemsetAsync(h->v.sums, 0, 8 * 2 * NSUMS, s);
  cudaMemsetAsync(h->v.hist, 0, 8 * 3 * h->v.nbins, s);
  cudaMemsetAsync(h->v.counters, 0, 8 * 2, s);
  return cuda_check(cudaGetLastError(), "stress reset");
}

// Time-averaged stresses (and the histogram) from the stress sums, sample
// counters and histogram read from the device (host arithmetic only).
static susp_status stress_from(const susp* h, const double* sums, const unsigned long long* cnt,
                               const double* hs, susp_stress_kind kind, double out[9], double* hist, int nbins) {
  if (hist && nbins == h->v.nbins) memcpy(hist, hs, 8 * 3 * (size_t)h->v.nbins);
  for (int k = 0; k < 9; ++k) out[k] = 0.0;
  if (cnt[0] == 0) return SUSP_OK;
  const double V = (double)h->v.nx * h->v.ny * h->v.nz;
  const double norm = 1.0 / (V * (double)cnt[0]);
  double visc[9], cont[9], rep[9], lub[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const int k = 3 * a + b, kt = 3 * b + a;
      visc[k] = norm * (sums[k] + 0.5 * (sums[9 + k] + sums[9 + kt]));
      cont[k] = -norm * sums[18 + k];
      rep[k] = -norm * sums[27 + k];
      lub[k] = norm * sums[36 + k];
    }
  switch (kind) {
    case SUSP_STRESS_VISCOUS: memcpy(out, visc, sizeof visc); break;
    case SUSP_STRESS_CONTACT: memcpy(out, cont, sizeof cont); break;
    case SUSP_STRESS_REPULSIVE: memcpy(out, rep, sizeof rep); break;
    case SUSP_STRESS_LUBRICATION: memcpy(out, lub, sizeof lub); break;
    case SUSP_STRESS_TOTAL:
      for (int k = 0; k < 9; ++k) out[k] = visc[k] + cont[k] + rep[k] + lub[k];
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

susp_status susp_stress(susp* h, susp_stress_kind kind, double out[9], double* hist, int nbins) {
  if (!h || !out) return fail(SUSP_EINVAL, "NULL argument");
  susp_status st = device_status(h);
  if (st) return st;
  double sums[NSUMS];
  unsigned long long cnt[2];
  std::vector<double> hs(3 * h->v.nbins);
  cudaMemcpy(sums, h->v.sums, sizeof sums, cudaMemcpyDeviceToHost);
  cudaMemcpy(cnt, h->v.counters, sizeof cnt, cudaMemcpyDeviceToHost);
  cudaMemcpy(hs.data(), h->v.hist, 8 * hs.size(), cudaMemcpyDeviceToHost);
  st = cuda_check(cudaGetLastError(), "read stress");
  if (st) return st;
  return stress_from(h, sums, cnt, hs.data(), kind, out, hist, nbins);
}

size_t susp_results_bytes(susp* h) { return h ? results_bytes(h->v.n, h->v.nbins) : 0; }

susp_status susp_read_results(susp* h, void* host_buf, size_t bytes, int async) {
  if (!h || !host_buf) return fail(SUSP_EINVAL, "NULL argument");
  if (async != 0 && async != 1) return fail(SUSP_EINVAL, "async must be 0 or 1");
  const size_t need = results_bytes(h->v.n, h->v.nbins);
  if (bytes < need) return fail(SUSP_EINVAL, "results buffer smaller than susp_results_bytes()");
  cudaStream_t s = stream_of(h);
  unsigned long long* stage = (unsigned long long*)(h->ws + h->L.res);
  const int words = (int)(need / 8);
  k_gather_results<<<(words + 255) / 256, 256, 0, s>>>(h->v, stage);
  cudaError_t e = cudaMemcpyAsync(host_buf, stage, need, cudaMemcpyDeviceToHost, s);
  susp_status st = cuda_check(e == cudaSuccess ? cudaGetLastError() : e, "read results");
  if (st || async) return st;
  st = cuda_check(cudaStreamSynchronize(s), "read results");
  if (st) return st;
  int err = 0;
  memcpy(&err, host_buf, sizeof(int));
  return err_status(err);
}

susp_status susp_results_particles(susp* h, const void* buf, double* pos, double* vel, double* omega) {
  if (!h || !buf) return fail(SUSP_EINVAL, "NULL argument");
  const char* b = (const char*)buf;
  int err = 0;
  memcpy(&err, b, sizeof(int));
  const size_t n3 = 24 * (size_t)h->v.n, o = res_parts(h->v.nbins);
  if (pos) memcpy(pos, b + o, n3);
  if (vel) memcpy(vel, b + o + n3, n3);
  if (omega) memcpy(omega, b + o + 2 * n3, n3);
  return err_status(err);
}

susp_status susp_results_stress(susp* h, const void* buf, susp_stress_kind kind, double out[9], double* hist,
                                int nbins) {
  if (!h || !buf || !out) return fail(SUSP_EINVAL, "NULL argument");
  const char* b = (const char*)buf;
  int err = 0;
  memcpy(&err, b, sizeof(int));
  susp_status st = err_status(err);
  if (st) return st;
  double sums[NSUMS];
  unsigned long long cnt[2];
  std::vector<double> hs(3 * h->v.nbins);
  memcpy(cnt, b + RES_CNT, sizeof cnt);
  memcpy(sums, b + RES_SUMS, sizeof sums);
  memcpy(hs.data(), b + res_hist(), 8 * hs.size());
  return stress_from(h, sums, cnt, hs.data(), kind, out, hist, nbins);
}

susp_status susp_moduli(susp* h, double* Gp, double* Gpp) {
  if (!h || !Gp || !Gpp) return fail(SUSP_EINVAL, "NULL argument");
  *Gp = *Gpp = 0.0;
  if (!h->have_shear || h->shear.kind != 1 || !(h->shear.gamma0 > 0.0))
    return fail(SUSP_ESTATE, "moduli need an oscillatory protocol with gamma0 > 0");
  susp_status st = device_status(h);
  if (st) return st;
  double sums[NSUMS];
  unsigned long long cnt[2];
  cudaMemcpy(sums, h->v.sums, sizeof sums, cudaMemcpyDeviceToHost);
  cudaMemcpy(cnt, h->v.counters, sizeof cnt, cudaMemcpyDeviceToHost);
  st = cuda_check(cudaGetLastError(), "read moduli sums");
  if (st) return st;
  if (cnt[0] == 0) return SUSP_OK;
  // the period integral times omega / pi is twice the window's time average
  const double V = (double)h->v.nx * h->v.ny * h->v.nz;
  const double norm = 1.0 / (V * (double)cnt[0]);
  *Gp = -2.0 * norm * sums[45] / h->shear.gamma0;
  *Gpp = 2.0 * norm * sums[46] / h->shear.gamma0;
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
  const void* fin = (read_proto(h).t & 1) ? h->v.fb : h->v.fa;
  st = cuda_check(cudaMemcpy(raw.data(), fin, raw.size(), cudaMemcpyDeviceToHost), "read populations");
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
  susp_status st = cuda_check(cudaStreamSynchronize(stream_of(h)), "sync");
  if (st) return st;
  void* fin = (read_proto(h).t & 1) ? h->v.fb : h->v.fa;
  st = cuda_check(cudaMemcpy(fin, raw.data(), raw.size(), cudaMemcpyHostToDevice), "write populations");
  if (st) return st;
  refresh_links(h);
  launch_plane_moments(h->prec, h->eng.B, h->eng.nplane, stream_of(h));
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
  const Proto pr = read_proto(h);
  st = cuda_check(cudaGetLastError(), "read protocol");
  if (st) return st;
  if (t) *t = pr.t;
  if (delta) *delta = pr.delta;
  return SUSP_OK;
}

susp_status susp_get_info(susp* h, susp_info* info) {
  if (!h || !info) return fail(SUSP_EINVAL, "NULL argument");
  const View& v = h->v;
  int dem = 0;
  if (v.move && v.n > 0) dem = (v.brute ? 0 : 4) + 1;
  info->dem_substeps = v.nsub;
  // collide-stream, particles (which end with the finalisation) or a
  // separate finalisation, node map + links
  info->launches_per_step = 1 + (dem ? dem : 1) + (v.n > 0 ? 3 : 0);
  info->brute_force_pairs = v.brute;
  info->ncell = v.ncell;
  info->workspace_bytes = h->L.total;
  const Engine& e = h->batch ? h->batch->eng : h->eng;
  info->overlap = e.ov_active ? 1 : 0;
  if (e.ov_active && dem) info->launches_per_step += 1;   // the separate finalisation
  return SUSP_OK;
}

// ------------------------------------------------------------ checkpoints

namespace {
struct CkptHeader {
  char magic[8];          // "SUSPCKP1"
  uint64_t total;         // workspace bytes
  int32_t nx, ny, nz, n, prec, have_shear;
  susp_shear shear;
};
}  // namespace

susp_status susp_save(susp* h, void* host_buf, size_t* bytes) {
  if (!h || !bytes) return fail(SUSP_EINVAL, "NULL argument");
  const size_t need = sizeof(CkptHeader) + h->L.total;
  if (!host_buf) { *bytes = need; return SUSP_OK; }
  if (*bytes < need) { *bytes = need; return fail(SUSP_ENOMEM, "checkpoint buffer too small"); }
  susp_status st = device_status(h);
  if (st) return st;
  CkptHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, "SUSPCKP1", 8);
  hd.total = h->L.total;
  hd.nx = h->p.nx; hd.ny = h->p.ny; hd.nz = h->p.nz; hd.n = h->p.n; hd.prec = h->prec;
  hd.have_shear = h->have_shear ? 1 : 0;
  hd.shear = h->shear;
  memcpy(host_buf, &hd, sizeof hd);
  st = cuda_check(cudaMemcpy((char*)host_buf + sizeof hd, h->ws, h->L.total, cudaMemcpyDeviceToHost), "save");
  if (st) return st;
  *bytes = need;
  return SUSP_OK;
}

susp_status susp_load(susp* h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf) return fail(SUSP_EINVAL, "NULL argument");
  CkptHeader hd;
  if (bytes < sizeof hd) return fail(SUSP_EINVAL, "checkpoint truncated");
  memcpy(&hd, host_buf, sizeof hd);
  if (memcmp(hd.magic, "SUSPCKP1", 8) != 0) return fail(SUSP_EINVAL, "not a checkpoint");
  if (hd.total != h->L.total || hd.nx != h->p.nx || hd.ny != h->p.ny || hd.nz != h->p.nz || hd.n != h->p.n ||
      hd.prec != h->prec)
    return fail(SUSP_EINVAL, "checkpoint made for other parameters");
  if (bytes < sizeof hd + hd.total) return fail(SUSP_EINVAL, "checkpoint truncated");
  cudaStream_t s = stream_of(h);
  susp_status st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (st) return st;
  st = cuda_check(cudaMemcpy(h->ws, (const char*)host_buf + sizeof hd, hd.total, cudaMemcpyHostToDevice), "load");
  if (st) return st;
  // the one-box descriptor holds device addresses of this workspace
  Engine& e = h->eng;
  std::vector<int> tabs;
  Engine tmp;
  tmp.prec = h->prec;
  tmp.tile_lg = e.tile_lg;
  eng_tables(tmp, std::vector<const View*>{&h->v}, tabs);
  st = cuda_check(cudaMemcpy(h->ws + h->L.views, &h->v, sizeof(View), cudaMemcpyHostToDevice), "load view");
  if (st) return st;
  // so do the tensor maps: the checkpoint may come from another box's workspace
  if (h->v.tmap) {
    st = cuda_check(cudaMemcpy(h->ws + h->L.tmap, h->maps.data(), h->maps.size(), cudaMemcpyHostToDevice),
                    "load tensor maps");
    if (st) return st;
  }
  st = cuda_check(cudaMemcpy(h->ws + h->L.tabs, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice), "load tables");
  if (st) return st;
  (void)e;
  h->have_shear = hd.have_shear != 0;
  h->shear = hd.shear;
  if (h->p.n > 0) {
    std::vector<double> r(h->p.n);
    st = cuda_check(cudaMemcpy(r.data(), h->v.rad, 8 * r.size(), cudaMemcpyDeviceToHost), "load radii");
    if (st) return st;
    h->radius = r;
  }
  return device_status(h);
}

susp_status susp_profile(susp* h, int enable) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  return eng_profile(h->eng, enable);
}

susp_status susp_profile_read(susp* h, double* ms_total, int* launches) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  return eng_profile_read(h->eng, ms_total, launches);
}

susp_status susp_profile_stages(susp* h, double* ms, int* steps) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  return eng_profile_stages(h->eng, ms, steps);
}

susp_status susp_set_graphs(susp* h, int enable) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  susp_status st = cuda_check(cudaStreamSynchronize(h->eng.stream), "sync");
  if (st) return st;
  eng_drop_graphs(h->eng);
  h->eng.use_graphs = enable != 0;
  return SUSP_OK;
}

susp_status susp_tune(susp* h, int* tile_rows, int* blocks_per_sm, double* us) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  if (h->batch) return fail(SUSP_ESTATE, "box is attached to a batch: tune the batch");
  return eng_tune(h->eng, std::vector<const View*>{&h->v}, h->ws + h->L.tabs, tile_rows, blocks_per_sm, us);
}

susp_status susp_set_launch_shape(susp* h, int tile_rows, int blocks_per_sm, int staged) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  if (h->batch) return fail(SUSP_ESTATE, "box is attached to a batch: set the batch's shape");
  return eng_set_shape(h->eng, std::vector<const View*>{&h->v}, h->ws + h->L.tabs, tile_rows, blocks_per_sm,
                       staged);
}

susp_status susp_set_overlap(susp* h, int enable) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  if (h->batch) return fail(SUSP_ESTATE, "box is attached to a batch: set the batch's overlap");
  return eng_set_overlap(h->eng, std::vector<const View*>{&h->v}, h->ws + h->L.tabs, enable);
}

susp_status susp_get_launch_shape(susp* h, int* tile_rows, int* blocks_per_sm, int* staged) {
  if (!h) return fail(SUSP_EINVAL, "NULL handle");
  eng_get_shape(h->batch ? h->batch->eng : h->eng, tile_rows, blocks_per_sm, staged);
  return SUSP_OK;
}

void susp_destroy(susp* h) {
  if (!h) return;
  if (h->batch) susp_batch_detach(h->batch, h);
  eng_release(h->eng);
  delete h;
}

// ------------------------------------------------------------ batches

size_t susp_batch_workspace_bytes(int max_boxes) {
  if (max_boxes < 1) { g_err = "max_boxes must be >= 1"; return 0; }
  return al(sizeof(View) * (size_t)max_boxes) + al(4 * sizeof(int) * (size_t)(max_boxes + 1)) +
         al(sizeof(int) * (size_t)max_boxes);
}

susp_status susp_batch_create(int max_boxes, void* dev_workspace, size_t bytes, void* cuda_stream,
                              susp_batch** out) {
  if (out) *out = nullptr;
  if (!out) return fail(SUSP_EINVAL, "out is NULL");
  if (max_boxes < 1) return fail(SUSP_EINVAL, "max_boxes must be >= 1");
  if (!dev_workspace || ((uintptr_t)dev_workspace & 255)) return fail(SUSP_EINVAL, "workspace NULL or not 256-byte aligned");
  if (bytes < susp_batch_workspace_bytes(max_boxes)) return fail(SUSP_ENOMEM, "workspace smaller than susp_batch_workspace_bytes()");
  if (!cuda_stream) return fail(SUSP_EINVAL, "a batch needs its own (non-default) stream");
  susp_batch* b = new susp_batch();
  b->max_boxes = max_boxes;
  b->prec = -1;
  b->ws = (char*)dev_workspace;
  b->eng.stream = (cudaStream_t)cuda_stream;
  return (*out = b, SUSP_OK);
}

// Upload the views and prefix tables of the attached boxes and reset the
// captured graphs (the launch shapes change with the membership).
static susp_status batch_rebuild(susp_batch* b) {
  Engine& e = b->eng;
  susp_status st = cuda_check(cudaStreamSynchronize(e.stream), "sync");
  if (st) return st;
  eng_drop_graphs(e);
  const int nb = (int)b->boxes.size();
  if (nb == 0) { e.nbox = 0; b->prec = -1; return SUSP_OK; }
  e.prec = b->prec;
  std::vector<const View*> vs;
  std::vector<View> hv;
  for (susp* h : b->boxes) { vs.push_back(&h->v); hv.push_back(h->v); }
  std::vector<int> tabs;
  eng_tables(e, vs, tabs);
  char* views = b->ws;
  char* tp = b->ws + al(sizeof(View) * (size_t)b->max_boxes);
  eng_bind(e, views, tp, nb);
  cudaMemcpyAsync(views, hv.data(), sizeof(View) * nb, cudaMemcpyHostToDevice, e.stream);
  cudaMemcpyAsync(tp, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, e.stream);
  return cuda_check(cudaStreamSynchronize(e.stream), "upload batch tables");
}

susp_status susp_batch_attach(susp_batch* b, susp* h) {
  if (!b || !h) return fail(SUSP_EINVAL, "NULL argument");
  if (h->batch) return fail(SUSP_ESTATE, "box is already attached to a batch");
  if ((int)b->boxes.size() >= b->max_boxes) return fail(SUSP_ENOMEM, "batch is full");
  if (b->prec >= 0 && b->prec != h->prec) return fail(SUSP_EINVAL, "boxes of one batch share the storage precision");
  if (!h->have_shear) return fail(SUSP_ESTATE, "set the box's shear protocol (susp_step with nsteps = 0) first");
  susp_status st = cuda_check(cudaStreamSynchronize(h->eng.stream), "sync box");
  if (st) return st;
  b->prec = h->prec;
  b->boxes.push_back(h);
  h->batch = b;
  st = batch_rebuild(b);
  if (st) { b->boxes.pop_back(); h->batch = nullptr; batch_rebuild(b); }
  return st;
}

susp_status susp_batch_detach(susp_batch* b, susp* h) {
  if (!b || !h) return fail(SUSP_EINVAL, "NULL argument");
  auto it = std::find(b->boxes.begin(), b->boxes.end(), h);
  if (it == b->boxes.end()) return fail(SUSP_ESTATE, "box is not attached to this batch");
  susp_status st = cuda_check(cudaStreamSynchronize(b->eng.stream), "sync batch");
  b->boxes.erase(it);
  h->batch = nullptr;
  susp_status st2 = batch_rebuild(b);
  return st ? st : st2;
}

int susp_batch_size(const susp_batch* b) { return b ? (int)b->boxes.size() : 0; }

susp_status susp_batch_step(susp_batch* b, int nsteps) {
  if (!b || nsteps < 0) return fail(SUSP_EINVAL, "bad argument to susp_batch_step");
  if (b->boxes.empty()) return SUSP_OK;
  return eng_step(b->eng, nsteps);
}

susp_status susp_batch_tune(susp_batch* b, int* tile_rows, int* blocks_per_sm, double* us) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  if (b->boxes.empty()) return fail(SUSP_ESTATE, "no box attached");
  std::vector<const View*> vs;
  for (susp* h : b->boxes) vs.push_back(&h->v);
  return eng_tune(b->eng, vs, b->ws + al(sizeof(View) * (size_t)b->max_boxes), tile_rows, blocks_per_sm, us);
}

susp_status susp_batch_set_launch_shape(susp_batch* b, int tile_rows, int blocks_per_sm, int staged) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  std::vector<const View*> vs;
  for (susp* h : b->boxes) vs.push_back(&h->v);
  return eng_set_shape(b->eng, vs, b->ws + al(sizeof(View) * (size_t)b->max_boxes), tile_rows, blocks_per_sm,
                       staged);
}

susp_status susp_batch_set_overlap(susp_batch* b, int enable) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  std::vector<const View*> vs;
  for (susp* h : b->boxes) vs.push_back(&h->v);
  return eng_set_overlap(b->eng, vs, b->ws + al(sizeof(View) * (size_t)b->max_boxes), enable);
}

susp_status susp_batch_get_overlap(susp_batch* b, int* overlap) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  if (overlap) *overlap = b->eng.ov_active ? 1 : 0;
  return SUSP_OK;
}

susp_status susp_batch_get_launch_shape(susp_batch* b, int* tile_rows, int* blocks_per_sm, int* staged) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  eng_get_shape(b->eng, tile_rows, blocks_per_sm, staged);
  return SUSP_OK;
}

susp_status susp_batch_profile(susp_batch* b, int enable) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  return eng_profile(b->eng, enable);
}

susp_status susp_batch_profile_read(susp_batch* b, double* ms_total, int* launches) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  return eng_profile_read(b->eng, ms_total, launches);
}

susp_status susp_batch_errors(susp_batch* b, int* status, int n) {
  if (!b || (!status && n > 0)) return fail(SUSP_EINVAL, "NULL argument");
  const int nb = (int)b->boxes.size();
  if (n < nb) return fail(SUSP_EINVAL, "status array shorter than the batch");
  if (nb == 0) return SUSP_OK;
  Engine& e = b->eng;
  int* dev = (int*)(b->ws + al(sizeof(View) * (size_t)b->max_boxes) +
                    al(4 * sizeof(int) * (size_t)(b->max_boxes + 1)));
  k_gather_err<<<(nb + 127) / 128, 128, 0, e.stream>>>(e.B, dev);
  std::vector<int> err(nb);
  susp_status st = cuda_check(cudaMemcpyAsync(err.data(), dev, sizeof(int) * nb, cudaMemcpyDeviceToHost,
                                              e.stream), "read error words");
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(e.stream), "sync batch");
  if (st) return st;
  const std::string keep = g_err;
  for (int k = 0; k < nb; ++k) status[k] = (int)err_status(err[k]);
  g_err = keep;
  return SUSP_OK;
}

susp_status susp_batch_profile_stages(susp_batch* b, double* ms, int* steps) {
  if (!b) return fail(SUSP_EINVAL, "NULL handle");
  return eng_profile_stages(b->eng, ms, steps);
}

void susp_batch_destroy(susp_batch* b) {
  if (!b) return;
  if (b->eng.stream) cudaStreamSynchronize(b->eng.stream);
  for (susp* h : b->boxes) h->batch = nullptr;
  b->boxes.clear();
  eng_release(b->eng);
  delete b;
}

}  // extern "C"
