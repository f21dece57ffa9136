// lclb_api.cu -- the C ABI of include/lc_lb.h: handles, device memory, the
// per-step launch sequence (captured once in a CUDA graph and replayed),
// geometry and boundary-link construction, exports, FP64 diagnostics, the
// relaxation driver, batches of boxes and the tile autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lc_lb.h"
#include "lclb_internal.h"

using namespace lclb;

struct Group;

namespace {

struct Allocator {
  lc_alloc_fn alloc = nullptr;
  lc_free_fn free = nullptr;
  void* ctx = nullptr;
};
Allocator g_alloc;
std::mutex g_mu;
thread_local std::string g_err;

struct TileCfg {
  int ty = 4, zc = 16, persistent = 0;
};

constexpr int NPHASE = 6;
// partial-sum doubles per tile of each phase
constexpr int PART_WIDTH[NPHASE] = {1, 4, 2, 1, 1, 1};

struct Phase {
  TileCfg cfg;
  int4* d_tiles = nullptr;
  int ntiles = 0;
  int grid = 0;
  std::vector<int> start, count;  // per box
  double* d_part = nullptr;
  size_t part_cap = 0;
};

// Partial records per tile: the Q update (phase 2) writes one per warp, TY per tile.
inline int part_records(const Phase& P, int k) { return k == 2 ? P.cfg.ty : 1; }

struct Mem {
  std::vector<std::pair<void*, cudaStream_t>> blocks;
  void* get(size_t bytes, cudaStream_t s, Allocator& al) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (al.alloc) {
      p = al.alloc(bytes, (void*)s, al.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) blocks.push_back({p, s});
    return p;
  }
  void put(void* p, Allocator& al) {
    for (size_t k = 0; k < blocks.size(); ++k)
      if (blocks[k].first == p) {
        if (al.free) al.free(p, (void*)blocks[k].second, al.ctx);
        else cudaFree(p);
        blocks.erase(blocks.begin() + (long)k);
        return;
      }
  }
  void release(Allocator& al) {
    for (auto& b : blocks) {
      if (al.free) al.free(b.first, (void*)b.second, al.ctx);
      else cudaFree(b.first);
    }
    blocks.clear();
  }
};

}  // namespace

struct lc_lb {
  Group* g = nullptr;
  int index = 0;
  bool owns_group = false;
  lc_grid grid{};
  lc_params params{};
  DevBox hb{};                          // host copy of the device descriptor
  std::vector<DevColloid> col;          // host-side configuration of the colloids
  int nlinks = 0;
  int* def = nullptr;                   // defect analytics: parent, comp, list (N each), block counts, total, error
  size_t def_cap = 0;
  std::string err;
};

struct Group {
  int prec = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Allocator al;
  Mem mem;
  std::vector<lc_lb*> boxes;
  DevBox* d_boxes = nullptr;
  // 0 force (diagnostics/export; split variant), 1 lb (split variant), 2 lc,
  // 3 fused force+lb (fused variant), 4 stress, 5 lb from stored stress (stored variant)
  Phase ph[NPHASE];
  cudaStream_t side = nullptr;   // second stream: link momentum exchange runs beside the Q update
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Step variant: 0 = fused stress/force/LB kernel; 1 = split: the stress/
  // force kernel and the LB kernel run concurrently in z slabs on two streams
  // (LB slab s waits for force slab s only); 2 = stored: H and P stored once
  // per node, then the LB kernel takes the face divergence of the stored P;
  // 3 = dataflow: the whole step (stored-stress kernels, Q update, link
  // exchange, colloid update) as one persistent launch k_step.
  int variant = 0;
  TileCfg step_cfg{4, 8, 0};        // dataflow: tile height and depth
  StepItem* d_items = nullptr;      // dataflow work list
  int nitems = 0, items_cap = 0;
  unsigned* d_sync = nullptr;       // item counter and completion counters
  int nsync = 0, sync_cap = 0;
  int* d_err = nullptr;             // set by k_step when a wait gave up
  int step_grid = 0;
  int slab = 0;                              // slab thickness in z (0: whole box)
  cudaStream_t side2 = nullptr;
  std::vector<cudaEvent_t> ev_slab;
  cudaEvent_t ev_lb = nullptr;
  std::vector<int2> chunk_f, chunk_lb;       // (first tile, count) per slab, force and LB phases
  int2* d_chunks = nullptr;
  int nchunks = 0, chunk_cap = 0;
  int2* d_mob = nullptr;        // (box, colloid) of every mobile colloid
  int nmob = 0, mob_cap = 0;
  double* d_scratch = nullptr;  // FP64 export buffer
  size_t scratch_cap = 0;
  double* d_red = nullptr;      // reduction outputs
  double* h_red = nullptr;      // pinned
  int* d_iwork = nullptr;       // link-build block sums
  size_t iwork_cap = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool dirty = true, tuned = false;
  int graph_kernels = 0;  // kernel nodes of the captured step
  int nsm = 0;
  int dev = 0;            // the device current when the group was created
  std::string err;
};

struct lc_lb_batch {
  Group* g = nullptr;
  std::string err;
};

namespace {

int fail(std::string* dst, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (dst) *dst = buf;
  g_err = buf;
  return code;
}

#define CK(call, dst)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(dst, LC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t tsize(int prec) { return prec == LC_FP64 ? 8 : 4; }

double bulk_q(double gam) {
  double t = 1.0 - 8.0 / (3.0 * gam);
  return t < 0.0 ? 0.0 : 0.25 + 0.75 * std::sqrt(t);
}

void* galloc(Group* g, size_t bytes) { return g->mem.get(bytes, g->stream, g->al); }

// Tile width in x of phase k for box b: 64 for the two-node paths of the
// stored-stress kernel and of the Q update (FP32 boxes of even width), else 32.
int tile_width(Group* g, int k, int b) { return ((k == 2 || k == 4) && g->boxes[b]->hb.pair) ? 64 : 32; }

// Tile list of one phase for every box of the group.
int build_phase(Group* g, int k) {
  Phase& P = g->ph[k];
  std::vector<int4> tl;
  P.start.assign(g->boxes.size(), 0);
  P.count.assign(g->boxes.size(), 0);
  for (size_t b = 0; b < g->boxes.size(); ++b) {
    const lc_grid& G = g->boxes[b]->grid;
    const int xs = tile_width(g, k, (int)b);
    P.start[b] = (int)tl.size();
    for (int z = 0; z < G.nz; z += P.cfg.zc)
      for (int y = 0; y < G.ny; y += P.cfg.ty)
        for (int x = 0; x < G.nx; x += xs) tl.push_back(make_int4((int)b, x, y, z));
    P.count[b] = (int)tl.size() - P.start[b];
  }
  if (P.d_tiles) g->mem.put(P.d_tiles, g->al);
  P.ntiles = (int)tl.size();
  P.d_tiles = (int4*)galloc(g, sizeof(int4) * tl.size());
  if (!P.d_tiles) return fail(&g->err, LC_ERR_OOM, "tile list allocation failed");
  CK(cudaMemcpyAsync(P.d_tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice, g->stream), &g->err);
  const size_t need = (size_t)PART_WIDTH[k] * tl.size() * part_records(P, k);
  if (need > P.part_cap) {
    if (P.d_part) g->mem.put(P.d_part, g->al);
    P.d_part = (double*)galloc(g, sizeof(double) * need);
    if (!P.d_part) return fail(&g->err, LC_ERR_OOM, "partials allocation failed");
    P.part_cap = need;
    CK(cudaMemsetAsync(P.d_part, 0, sizeof(double) * need, g->stream), &g->err);
  }
  P.grid = P.cfg.persistent ? std::min(P.ntiles, g->nsm * P.cfg.persistent) : P.ntiles;
  if (P.grid < 1) P.grid = 1;
  g->dirty = true;
  return LC_OK;
}

Launch phase_launch(Group* g, int k, int box = -1) {
  Phase& P = g->ph[k];
  Launch L;
  L.boxes = g->d_boxes;
  L.zc = P.cfg.zc;
  L.ty = P.cfg.ty;
  L.stream = g->stream;
  if (box < 0) {
    L.tiles = P.d_tiles;
    L.ntiles = P.ntiles;
    L.grid = P.grid;
  } else {
    L.tiles = P.d_tiles + P.start[box];
    L.ntiles = P.count[box];
    L.grid = P.count[box];
  }
  return L;
}

int upload_box(Group* g, lc_lb* h) {
  CK(cudaMemcpyAsync(g->d_boxes + h->index, &h->hb, sizeof(DevBox), cudaMemcpyHostToDevice, g->stream), &h->err);
  g->dirty = true;
  return LC_OK;
}

// Link chunks (box, first link) covering every box's link capacity.
int build_chunks(Group* g) {
  std::vector<int2> ch;
  for (size_t b = 0; b < g->boxes.size(); ++b) {
    const lc_lb* h = g->boxes[b];
    for (int s = 0; s < h->hb.nlinks_cap; s += LINK_CHUNK) ch.push_back(make_int2((int)b, s));
  }
  if ((int)ch.size() > g->chunk_cap) {
    if (g->d_chunks) g->mem.put(g->d_chunks, g->al);
    g->chunk_cap = (int)ch.size() + 64;
    g->d_chunks = (int2*)galloc(g, sizeof(int2) * g->chunk_cap);
    if (!g->d_chunks) return fail(&g->err, LC_ERR_OOM, "link chunk allocation failed");
  }
  g->nchunks = (int)ch.size();
  if (!ch.empty())
    CK(cudaMemcpyAsync(g->d_chunks, ch.data(), sizeof(int2) * ch.size(), cudaMemcpyHostToDevice, g->stream), &g->err);
  g->dirty = true;
  return LC_OK;
}

int ensure_scratch(Group* g, size_t doubles) {
  if (doubles <= g->scratch_cap) return LC_OK;
  if (g->d_scratch) g->mem.put(g->d_scratch, g->al);
  g->d_scratch = (double*)galloc(g, sizeof(double) * doubles);
  if (!g->d_scratch) return fail(&g->err, LC_ERR_OOM, "scratch allocation failed");
  g->scratch_cap = doubles;
  return LC_OK;
}

int ensure_iwork(Group* g, size_t ints) {
  if (ints <= g->iwork_cap) return LC_OK;
  if (g->d_iwork) g->mem.put(g->d_iwork, g->al);
  g->d_iwork = (int*)galloc(g, sizeof(int) * ints);
  if (!g->d_iwork) return fail(&g->err, LC_ERR_OOM, "work allocation failed");
  g->iwork_cap = ints;
  return LC_OK;
}

int check_params(const lc_grid* G, const lc_params* p, std::string* err) {
  if (!G || !p) return fail(err, LC_ERR_ARG, "null grid or params");
  if (G->nx < 1 || G->ny < 1 || G->nz < 1) return fail(err, LC_ERR_ARG, "box dimensions must be >= 1");
  if ((long long)G->nx * G->ny * G->nz >= (1LL << 31) - 1) return fail(err, LC_ERR_ARG, "box too large (N >= 2^31)");
  if (!(p->tau > 0.5)) return fail(err, LC_ERR_ARG, "tau must exceed 1/2");
  if (p->precision != LC_FP32 && p->precision != LC_FP64) return fail(err, LC_ERR_ARG, "unknown precision");
  if (!(p->rho0 > 0.0)) return fail(err, LC_ERR_ARG, "rho0 must be positive");
  return LC_OK;
}

int write_state(Group* g, lc_lb* h, int pre_valid) {
  DevState st{};
  st.fpar = 0;
  st.qpar = 0;
  st.pre_valid = pre_valid;
  st.cstep = -1;
  CK(cudaMemcpyAsync(h->hb.st, &st, sizeof(st), cudaMemcpyHostToDevice, g->stream), &h->err);
  return LC_OK;
}

template <typename T>
void fill_phys(PhysT<T>& o, const DevParams& p) {
  o.rho0 = (T)p.rho0;
  o.omega = (T)(1.0 / p.tau);
  o.pref = (T)(1.0 - 0.5 / p.tau);
  o.A0 = (T)p.A0; o.gamma = (T)p.gamma; o.K = (T)p.K; o.q0 = (T)p.q0; o.xi = (T)p.xi; o.Gamma = (T)p.Gamma;
  o.S0 = (T)p.S0;
  for (int a = 0; a < 3; ++a) o.g[a] = (T)p.g[a];
}

// Allocate and initialise one box inside group g.
int make_box(Group* g, const lc_grid* G, const lc_params* p, lc_lb* h) {
  h->grid = *G;
  h->params = *p;
  DevBox& B = h->hb;
  memset(&B, 0, sizeof(B));
  B.nx = G->nx; B.ny = G->ny; B.nz = G->nz; B.wall_z = G->wall_z ? 1 : 0;
  B.pair = pair_width(G->nx, g->prec == LC_FP32) ? 1 : 0;
  B.N = G->nx * G->ny * G->nz;
  const size_t N = (size_t)B.N, ts = tsize(g->prec);
  B.p.rho0 = p->rho0; B.p.tau = p->tau; B.p.A0 = p->A0; B.p.gamma = p->gamma; B.p.K = p->K; B.p.q0 = p->q0;
  B.p.xi = p->xi; B.p.Gamma = p->Gamma; B.p.S0 = p->S0 > 0.0 ? p->S0 : bulk_q(p->gamma);
  for (int a = 0; a < 3; ++a) B.p.g[a] = p->body_force[a];
  B.p.lc_on = p->lc_enabled ? 1 : 0;
  B.p.flow_on = p->flow_enabled ? 1 : 0;
  fill_phys(B.pf, B.p);
  fill_phys(B.pd, B.p);
  for (int k = 0; k < 2; ++k) {
    B.f[k] = galloc(g, NQ * N * ts);
    B.Q[k] = galloc(g, 5 * N * ts);
    if (g->prec == LC_FP32) {
      B.Qlo[k] = (__nv_bfloat16*)galloc(g, 5 * N * sizeof(__nv_bfloat16));
      if (!B.Qlo[k]) return fail(&h->err, LC_ERR_OOM, "device allocation failed for a %dx%dx%d box", G->nx, G->ny, G->nz);
    }
  }
  B.u = galloc(g, 3 * N * ts);
  B.F = galloc(g, 3 * N * ts);
  B.H = galloc(g, 5 * N * ts);
  B.P = galloc(g, 9 * N * ts);
  B.mask = (uint8_t*)galloc(g, N);
  B.col = (DevColloid*)galloc(g, sizeof(DevColloid) * MAXCOL);
  B.st = (DevState*)galloc(g, sizeof(DevState));
  B.gerr = g->d_err;
  B.nlinks = (int*)galloc(g, sizeof(int));
  if (!B.f[0] || !B.f[1] || !B.Q[0] || !B.Q[1] || !B.u || !B.F || !B.H || !B.P || !B.mask || !B.col || !B.st ||
      !B.nlinks)
    return fail(&h->err, LC_ERR_OOM, "device allocation failed for a %dx%dx%d box", G->nx, G->ny, G->nz);
  cudaStream_t s = g->stream;
  for (int k = 0; k < 2; ++k) {
    CK(cudaMemsetAsync(B.f[k], 0, NQ * N * ts, s), &h->err);
    if (B.Qlo[k]) CK(cudaMemsetAsync(B.Qlo[k], 0, 5 * N * sizeof(__nv_bfloat16), s), &h->err);
  }
  CK(cudaMemsetAsync(B.u, 0, 3 * N * ts, s), &h->err);
  CK(cudaMemsetAsync(B.F, 0, 3 * N * ts, s), &h->err);
  CK(cudaMemsetAsync(B.H, 0, 5 * N * ts, s), &h->err);
  CK(cudaMemsetAsync(B.P, 0, 9 * N * ts, s), &h->err);
  CK(cudaMemsetAsync(B.mask, 0, N, s), &h->err);
  CK(cudaMemsetAsync(B.col, 0, sizeof(DevColloid) * MAXCOL, s), &h->err);
  CK(cudaMemsetAsync(B.nlinks, 0, sizeof(int), s), &h->err);
  int rc = write_state(g, h, 1);
  if (rc) return rc;
  rc = upload_box(g, h);
  if (rc) return rc;
  const double n[3] = {0.0, 0.0, 1.0};
  CK(launch_geometry(g->d_boxes, h->index, B.N, s), &h->err);
  CK(launch_init_q(g->prec, g->d_boxes, h->index, B.N, 0, n, 0.0, 0ULL, s), &h->err);
  return LC_OK;
}

Group* new_group(int prec, void* stream, int nboxes, std::string* err) {
  Group* g = new Group();
  g->prec = prec;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g->al = g_alloc;
  }
  if (stream) {
    g->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      fail(err, LC_ERR_CUDA, "cannot create a stream");
      delete g;
      return nullptr;
    }
    g->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_lb, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    fail(err, LC_ERR_CUDA, "cannot create the side stream");
    delete g;
    return nullptr;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  g->dev = dev;
  cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (g->nsm <= 0) g->nsm = 1;
  g->d_boxes = (DevBox*)galloc(g, sizeof(DevBox) * std::max(1, nboxes));
  g->d_red = (double*)galloc(g, sizeof(double) * 64);
  g->d_err = (int*)galloc(g, sizeof(int) * 4);
  if (g->d_err) cudaMemsetAsync(g->d_err, 0, sizeof(int) * 4, g->stream);
  if (!g->d_boxes || !g->d_red || !g->d_err || cudaMallocHost(&g->h_red, sizeof(double) * 64) != cudaSuccess) {
    fail(err, LC_ERR_OOM, "group allocation failed");
    g->mem.release(g->al);
    if (g->own_stream) cudaStreamDestroy(g->stream);
    delete g;
    return nullptr;
  }
  return g;
}

void free_group(Group* g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->mem.release(g->al);
  if (g->h_red) cudaFreeHost(g->h_red);
  if (g->side) {
    cudaStreamSynchronize(g->side);
    cudaStreamDestroy(g->side);
  }
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  if (g->side2) {
    cudaStreamSynchronize(g->side2);
    cudaStreamDestroy(g->side2);
  }
  if (g->ev_lb) cudaEventDestroy(g->ev_lb);
  for (cudaEvent_t e : g->ev_slab) cudaEventDestroy(e);
  if (g->own_stream) cudaStreamDestroy(g->stream);
  for (lc_lb* h : g->boxes) delete h;
  delete g;
}

// ---- autotuning -------------------------------------------------------------
using TuneKey = std::tuple<long long, int>;  // (sum of box signature, precision)
std::map<TuneKey, std::vector<TileCfg>> g_tune_cache;

TuneKey tune_key(Group* g) {
  long long sig = 1469598103934665603LL;
  for (lc_lb* h : g->boxes) {
    sig = sig * 1099511628211LL + h->grid.nx;
    sig = sig * 1099511628211LL + h->grid.ny;
    sig = sig * 1099511628211LL + h->grid.nz;
    sig = sig * 1099511628211LL + h->grid.wall_z;
  }
  return TuneKey(sig, g->prec);
}

// Optional file cache (LCLB_TUNE_CACHE): one line per entry,
// "signature precision" and NCFG triples "ty zc persistent" (fused, lc,
// force, lb, (variant, slab, 0), stress, lb-from-stress, dataflow step);
// lines of another length are skipped.
constexpr int NCFG = 8;
void tune_file_load() {
  const char* path = getenv("LCLB_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    long long sig;
    int prec, v[3 * NCFG], used = 0, n = 0;
    if (sscanf(line, "%lld %d%n", &sig, &prec, &used) != 2) continue;
    const char* q = line + used;
    while (n < 3 * NCFG) {
      int adv = 0;
      if (sscanf(q, "%d%n", &v[n], &adv) != 1) break;
      q += adv;
      ++n;
    }
    int extra = 0;
    if (n != 3 * NCFG || sscanf(q, "%d", &extra) == 1) continue;
    std::vector<TileCfg> c(NCFG);
    for (int k = 0; k < NCFG; ++k) c[k] = TileCfg{v[3 * k], v[3 * k + 1], v[3 * k + 2]};
    g_tune_cache[TuneKey(sig, prec)] = c;
  }
  fclose(f);
}

void tune_file_store(const TuneKey& key, const std::vector<TileCfg>& c) {
  const char* path = getenv("LCLB_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%lld %d", std::get<0>(key), std::get<1>(key));
  for (int k = 0; k < NCFG; ++k) fprintf(f, " %d %d %d", c[k].ty, c[k].zc, c[k].persistent);
  fprintf(f, "\n");
  fclose(f);
}

cudaError_t launch_phase(Group* g, int k, int mode, int box = -1) {
  Launch L = phase_launch(g, k, box);
  double* part = g->ph[k].d_part +
                 (box < 0 ? 0 : (size_t)g->ph[k].start[box] * PART_WIDTH[k] * part_records(g->ph[k], k));
  if (k == 0) return launch_force(g->prec, L, mode, part);
  if (k == 1) return launch_lb(g->prec, L, mode, part);
  if (k == 2) return launch_lc(g->prec, L, mode, part);
  if (k == 4) return launch_stress(g->prec, L, mode, part);
  if (k == 5) return launch_lbp(g->prec, L, mode, part);
  return launch_flb(g->prec, L, mode, part);
}

// Time every candidate tile shape of each phase on the group's own state (the
// phase kernels are idempotent between parity flips) and keep the fastest.
int build_chunks_slab(Group* g);
int enqueue_split(Group* g, int force_mode);

float time_ms(Group* g, cudaEvent_t e0, cudaEvent_t e1, int reps, int (*fn)(Group*, void*), void* arg, int* rc) {
  *rc = fn(g, arg);  // warm-up
  if (*rc) return 1e30f;
  if (cudaEventRecord(e0, g->stream) != cudaSuccess) return 1e30f;
  for (int r = 0; r < reps && !*rc; ++r) *rc = fn(g, arg);
  if (*rc || cudaEventRecord(e1, g->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / reps;
}

int tune_phase_fn(Group* g, void* arg) {
  const int k = *static_cast<int*>(arg);
  const int mode = k == 2 ? LC_RESID : 0;  // no colloid accumulation while tuning
  CK(launch_phase(g, k, mode), &g->err);
  return LC_OK;
}
int tune_split_fn(Group* g, void*) { return enqueue_split(g, 0); }
int tune_stored_fn(Group* g, void*) {
  CK(launch_phase(g, 4, 0), &g->err);
  CK(launch_phase(g, 5, 0), &g->err);
  return LC_OK;
}
cudaError_t launch_dataflow(Group* g, int commit);
int build_items(Group* g);
int tune_dataflow_fn(Group* g, void*) {
  CK(launch_dataflow(g, 0), &g->err);
  return LC_OK;
}

// Time every candidate tile shape of each phase kernel on the group's own
// state (the phase kernels are idempotent between parity flips), then the
// slab thickness of the split variant, then fused against split, and keep
// the fastest.
int autotune_group_inner(Group* g, std::string* desc);

// The LB kernels read f in place while the populations are pre-collision
// (just after initialisation or set_fields) and pull from the neighbours in
// every later step; tune on the pull path, then put each box's state back.
int autotune_group(Group* g, std::string* desc) {
  std::vector<DevState> saved(g->boxes.size());
  for (size_t b = 0; b < g->boxes.size(); ++b) {
    lc_lb* h = g->boxes[b];
    CK(cudaMemcpyAsync(&saved[b], h->hb.st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream), &g->err);
  }
  CK(cudaStreamSynchronize(g->stream), &g->err);
  for (size_t b = 0; b < g->boxes.size(); ++b) {
    if (!saved[b].pre_valid) continue;
    CK(cudaMemsetAsync(&g->boxes[b]->hb.st->pre_valid, 0, sizeof(int), g->stream), &g->err);
  }
  const int rc = autotune_group_inner(g, desc);
  for (size_t b = 0; b < g->boxes.size(); ++b)
    CK(cudaMemcpyAsync(g->boxes[b]->hb.st, &saved[b], sizeof(DevState), cudaMemcpyHostToDevice, g->stream), &g->err);
  CK(cudaStreamSynchronize(g->stream), &g->err);
  return rc;
}

int autotune_group_inner(Group* g, std::string* desc) {
  const int pers[3] = {0, 2, 4};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), &g->err);
  CK(cudaEventCreate(&e1), &g->err);
  char buf[256];
  std::string out;
  int rc = LC_OK;
  float best_phase[NPHASE] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
  const char* venv = getenv("LCLB_TUNE_VERBOSE");
  const bool verbose = venv && venv[0] == '1';
  // FP32 boxes: only the stored-stress kernels take the derivatives at nodes
  // next to a solid from the compensated Q (the colloid force needs them), so
  // the fused and split variants are not candidates there (LCLB_VARIANT still
  // forces them)
  const bool fp32 = g->prec == LC_FP32;
  for (int k : {3, 2, 0, 1, 4, 5}) {
    if (fp32 && (k == 3 || k == 1)) continue;
    TileCfg best = g->ph[k].cfg;
    const std::vector<int> tys = k == 3 ? std::vector<int>{4, 6, 8} : std::vector<int>{2, 4, 8};
    const std::vector<int> zcs =
        (k == 1 || k == 5) ? std::vector<int>{1, 2, 4, 8, 16} : std::vector<int>{2, 4, 8, 16, 32, 64};
    for (int ty : tys)
      for (int zc : zcs)
        for (int pp : pers) {
          g->ph[k].cfg = TileCfg{ty, zc, pp};
          if ((rc = build_phase(g, k))) return rc;
          int kk = k;
          const float ms = time_ms(g, e0, e1, 3, tune_phase_fn, &kk, &rc);
          if (rc) return rc;
          if (verbose) fprintf(stderr, "lclb tune phase %d ty=%d zc=%d pers=%d %.1f us\n", k, ty, zc, pp, 1000.f * ms);
          if (ms < best_phase[k]) {
            best_phase[k] = ms;
            best = g->ph[k].cfg;
          }
        }
    g->ph[k].cfg = best;
    if ((rc = build_phase(g, k))) return rc;
    snprintf(buf, sizeof(buf), "%s:ty=%d,zc=%d,pers=%d(%.1fus) ",
             k == 3 ? "flb" : (k == 2 ? "lc" : (k == 0 ? "force" : (k == 1 ? "lb" : (k == 4 ? "stress" : "lbp")))),
             best.ty, best.zc, best.persistent,
             1000.f * best_phase[k]);
    out += buf;
  }
  // split variant: slab thickness (multiples of both tile depths), 0 = whole box
  int maxnz = 1;
  for (lc_lb* h : g->boxes) maxnz = std::max(maxnz, h->grid.nz);
  const int a = g->ph[0].cfg.zc, b = g->ph[1].cfg.zc;
  int l = a;
  while (l % b) l += a;
  float best_split = 1e30f;
  int best_slab = 0;
  for (int m = 1; !fp32 && l * m <= maxnz; m *= 2) {
    g->slab = l * m;
    if ((rc = build_chunks_slab(g))) return rc;
    const float ms = time_ms(g, e0, e1, 3, tune_split_fn, nullptr, &rc);
    if (rc) return rc;
    if (verbose) fprintf(stderr, "lclb tune split slab=%d %.1f us\n", g->slab, 1000.f * ms);
    if (ms < best_split) {
      best_split = ms;
      best_slab = g->slab;
    }
  }
  g->slab = best_slab;
  if ((rc = build_chunks_slab(g))) return rc;
  const float stored = time_ms(g, e0, e1, 3, tune_stored_fn, nullptr, &rc);
  if (rc) return rc;
  if (verbose) fprintf(stderr, "lclb tune stored %.1f us\n", 1000.f * stored);
  g->variant = 0;
  float best_var = best_phase[3];
  if (best_split < best_var) {
    g->variant = 1;
    best_var = best_split;
  }
  if (stored < best_var || fp32) {
    g->variant = 2;
    best_var = stored;
  }
  // dataflow: the whole step as one launch, timed without committing it
  // (against the force + LB part plus the Q update of the classic variants)
  const float classic = best_var + best_phase[2];
  const TileCfg lc_cfg = g->ph[2].cfg;
  float best_df = 1e30f;
  TileCfg best_step = g->step_cfg;
  const char* dfenv = getenv("LCLB_DATAFLOW");
  if (!(dfenv && dfenv[0] == '0')) {
    for (int ty : {2, 4, 8})
      for (int zc : {4, 8, 16}) {
        g->step_cfg = TileCfg{ty, zc, 0};
        if ((rc = build_items(g))) return rc;
        const float ms = time_ms(g, e0, e1, 3, tune_dataflow_fn, nullptr, &rc);
        if (rc) return rc;
        if (verbose) fprintf(stderr, "lclb tune dataflow ty=%d zc=%d %.1f us\n", ty, zc, 1000.f * ms);
        if (ms < best_df) {
          best_df = ms;
          best_step = g->step_cfg;
        }
      }
  }
  g->step_cfg = best_step;
  if (best_df < classic) {
    g->variant = 3;
    g->ph[2].cfg = TileCfg{best_step.ty, best_step.zc, lc_cfg.persistent};
  } else {
    g->ph[2].cfg = lc_cfg;
  }
  if ((rc = build_phase(g, 2))) return rc;
  static const char* vname[4] = {"fused", "split", "stored", "dataflow"};
  snprintf(buf, sizeof(buf), "split(slab=%d,%.1fus) stored(%.1fus) classic+lc(%.1fus) dataflow(ty=%d,zc=%d,%.1fus) -> %s",
           best_slab, 1000.f * best_split, 1000.f * stored, 1000.f * classic, best_step.ty, best_step.zc,
           1000.f * best_df, vname[g->variant]);
  out += buf;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune_cache[tune_key(g)] = {g->ph[3].cfg, g->ph[2].cfg, g->ph[0].cfg, g->ph[1].cfg,
                                 TileCfg{g->variant, g->slab, 0}, g->ph[4].cfg, g->ph[5].cfg, g->step_cfg};
    tune_file_store(tune_key(g), g_tune_cache[tune_key(g)]);
  }
  g->tuned = true;
  g->dirty = true;
  if (desc) *desc = out;
  return LC_OK;
}

// LCLB_VARIANT=fused|split|stored|dataflow forces the variant of the step
// (the tile shapes stay tuned); used to run every variant through the same tests.
int apply_variant_override(Group* g) {
  const char* v = getenv("LCLB_VARIANT");
  if (!v || !v[0]) return LC_OK;
  const int want = !strcmp(v, "fused") ? 0
                   : !strcmp(v, "split") ? 1
                   : !strcmp(v, "stored") ? 2
                   : !strcmp(v, "dataflow") ? 3 : -1;
  if (want < 0) return fail(&g->err, LC_ERR_ARG, "LCLB_VARIANT must be fused, split, stored or dataflow (got %s)", v);
  if (want != g->variant) {
    g->variant = want;
    if (want == 3) {
      g->ph[2].cfg = TileCfg{g->step_cfg.ty, g->step_cfg.zc, g->ph[2].cfg.persistent};
      if (int rc = build_phase(g, 2)) return rc;
    }
    g->dirty = true;
  }
  return LC_OK;
}

int maybe_tune(Group* g) {
  if (g->tuned) return apply_variant_override(g);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    static bool loaded = false;
    if (!loaded) {
      tune_file_load();
      loaded = true;
    }
    auto it = g_tune_cache.find(tune_key(g));
    if (it != g_tune_cache.end()) {
      g->ph[3].cfg = it->second[0];
      g->ph[2].cfg = it->second[1];
      g->ph[0].cfg = it->second[2];
      g->ph[1].cfg = it->second[3];
      g->variant = it->second[4].ty;
      g->slab = it->second[4].zc;
      g->ph[4].cfg = it->second[5];
      g->ph[5].cfg = it->second[6];
      g->step_cfg = it->second[7];
      g->tuned = true;
    }
  }
  int rc = LC_OK;
  if (g->tuned) {
    if (g->variant == 3) g->ph[2].cfg = TileCfg{g->step_cfg.ty, g->step_cfg.zc, g->ph[2].cfg.persistent};
    for (int k = 0; k < NPHASE && !rc; ++k) rc = build_phase(g, k);
    if (!rc) rc = build_chunks_slab(g);
  } else {
    const char* env = getenv("LCLB_AUTOTUNE");
    if (env && env[0] == '0') {
      g->tuned = true;
      rc = build_chunks_slab(g);
    } else {
      rc = autotune_group(g, nullptr);
    }
  }
  return rc ? rc : apply_variant_override(g);
}

// ---- one step -----------------------------------------------------------------
// Slab chunks of the force (phase 0) and LB (phase 1) tile lists: tiles are
// ordered (box, z, y, x), so the tiles of box b with z0 in [s*slab,
// (s+1)*slab) are contiguous in both lists.
int build_chunks_slab(Group* g) {
  g->chunk_f.clear();
  g->chunk_lb.clear();
  const Phase& F = g->ph[0];
  const Phase& L = g->ph[1];
  for (size_t b = 0; b < g->boxes.size(); ++b) {
    const int nz = g->boxes[b]->grid.nz;
    const int sz = g->slab > 0 ? g->slab : nz;
    int fi = F.start[b], li = L.start[b];
    const int fe = F.start[b] + F.count[b], le = L.start[b] + L.count[b];
    const int zcF = F.cfg.zc, zcL = L.cfg.zc;
    const int tilesF = F.count[b] / ((nz + zcF - 1) / zcF), tilesL = L.count[b] / ((nz + zcL - 1) / zcL);
    for (int z = 0; z < nz; z += sz) {
      const int ze = std::min(nz, z + sz);
      const int nf = ((ze + zcF - 1) / zcF - (z + zcF - 1) / zcF) * tilesF;
      const int nl = ((ze + zcL - 1) / zcL - (z + zcL - 1) / zcL) * tilesL;
      g->chunk_f.push_back(make_int2(fi, nf));
      g->chunk_lb.push_back(make_int2(li, nl));
      fi += nf;
      li += nl;
    }
    if (fi != fe || li != le) return fail(&g->err, LC_ERR_STATE, "slab chunks do not cover the tile lists");
  }
  while (g->ev_slab.size() < g->chunk_f.size()) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), &g->err);
    g->ev_slab.push_back(e);
  }
  g->dirty = true;
  return LC_OK;
}

cudaError_t launch_range(Group* g, int k, int2 range, int mode, cudaStream_t st) {
  Phase& P = g->ph[k];
  Launch L;
  L.boxes = g->d_boxes;
  L.zc = P.cfg.zc;
  L.ty = P.cfg.ty;
  L.stream = st;
  L.tiles = P.d_tiles + range.x;
  L.ntiles = range.y;
  L.grid = P.cfg.persistent ? std::max(1, std::min(range.y, g->nsm * P.cfg.persistent)) : range.y;
  const int width = k == 0 ? 1 : 4;
  double* part = P.d_part + (size_t)range.x * width;
  return k == 0 ? launch_force(g->prec, L, mode, part) : launch_lb(g->prec, L, mode, part);
}

// Split variant of the force + LB part of a step (see Group::variant).
int enqueue_split(Group* g, int force_mode) {
  const size_t n = g->chunk_f.size();
  for (size_t c = 0; c < n; ++c) {
    if (g->chunk_f[c].y > 0) CK(launch_range(g, 0, g->chunk_f[c], force_mode, g->stream), &g->err);
    CK(cudaEventRecord(g->ev_slab[c], g->stream), &g->err);
  }
  for (size_t c = 0; c < n; ++c) {
    CK(cudaStreamWaitEvent(g->side2, g->ev_slab[c], 0), &g->err);
    if (g->chunk_lb[c].y > 0) CK(launch_range(g, 1, g->chunk_lb[c], 0, g->side2), &g->err);
  }
  CK(cudaEventRecord(g->ev_lb, g->side2), &g->err);
  CK(cudaStreamWaitEvent(g->stream, g->ev_lb, 0), &g->err);
  return LC_OK;
}

// ---- dataflow variant: work list of the persistent step kernel ---------------
// Per box b with nzc = ceil(nz / zc) chunks of zc planes and tpc tiles per
// chunk, counters (after sync[0], the item counter): stress, LB and Q update
// done per chunk (3 nzc), then all stress, all LB, all Q update and all link
// chunks done (4).  Chunks are visited in the order 0, nzc-1, 1, nzc-2, ...
// for a periodic box (the wrap neighbours of the first chunks come early) and
// 0, 1, ... between walls; at stage w a box contributes the stress tiles of
// its w-th chunk, the LB tiles of its (w-2)-th and the Q-update tiles of its
// (w-4)-th, its link chunks after its last LB chunk and its colloid update
// after its last Q-update chunk.  Every item then follows what it waits for.
int build_items(Group* g) {
  const int ty = g->step_cfg.ty, zc = g->step_cfg.zc;
  Phase& PL = g->ph[2];
  if (PL.cfg.ty != ty || PL.cfg.zc != zc) {
    PL.cfg.ty = ty;
    PL.cfg.zc = zc;
    if (int rc = build_phase(g, 2)) return rc;
  }
  const int nb = (int)g->boxes.size();
  // tiles per chunk row in x: stress (ntxs), LB (ntxl, always 32 wide), Q update (ntx)
  std::vector<int> base(nb), nzc(nb), ntx(nb), ntxs(nb), ntxl(nb), nty(nb), nlk(nb);
  int ncnt = 1, maxz = 0;
  for (int b = 0; b < nb; ++b) {
    const lc_lb* h = g->boxes[b];
    nzc[b] = (h->grid.nz + zc - 1) / zc;
    const int ws = tile_width(g, 4, b), wq = tile_width(g, 2, b);
    ntxs[b] = (h->grid.nx + ws - 1) / ws;
    ntxl[b] = (h->grid.nx + 31) / 32;
    ntx[b] = (h->grid.nx + wq - 1) / wq;
    nty[b] = (h->grid.ny + ty - 1) / ty;
    nlk[b] = (h->hb.nlinks_cap + LINK_CHUNK - 1) / LINK_CHUNK;
    base[b] = ncnt;
    ncnt += 3 * nzc[b] + 4;
    maxz = std::max(maxz, nzc[b]);
  }
  // an extra counter that nothing increments: LCLB_TEST_STALL=1 makes the
  // first LB item wait on it (a test of the bounded waits)
  const int never = ncnt++;
  const char* stall_env = getenv("LCLB_TEST_STALL");
  bool stall = stall_env && stall_env[0] == '1';
  std::vector<StepItem> it;
  auto chunk_of = [&](int b, int k) {
    const int n = nzc[b];
    if (g->boxes[b]->grid.wall_z) return k;
    return (k % 2 == 0) ? k / 2 : n - 1 - k / 2;
  };
  auto blank = [](int kind, int b) {
    StepItem I;
    I.kind = kind;
    I.box = b;
    I.x0 = I.y0 = I.z0 = I.part = 0;
    for (int k = 0; k < 4; ++k) I.wc[k] = -1, I.wt[k] = 0;
    I.dc[0] = I.dc[1] = -1;
    return I;
  };
  // counter of phase p (0 stress, 1 LB, 2 Q update) for chunk c of box b
  auto cnt = [&](int b, int p, int c) { return base[b] + p * nzc[b] + c; };
  auto neighbour_waits = [&](StepItem& I, int b, int p, int c) {
    const int n = nzc[b], tpc = (p == 0 ? ntxs[b] : (p == 1 ? ntxl[b] : ntx[b])) * nty[b];
    int k = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      int cc = c + dz;
      if (g->boxes[b]->grid.wall_z) {
        if (cc < 0 || cc >= n) continue;
      } else {
        cc = (cc + n) % n;
      }
      const int id = cnt(b, p, cc);
      bool dup = false;
      for (int j = 0; j < k; ++j) dup = dup || I.wc[j] == id;
      if (dup) continue;
      I.wc[k] = id;
      I.wt[k] = tpc;
      ++k;
    }
  };
  auto tiles = [&](int kind, int b, int c) {
    const lc_grid& G = g->boxes[b]->grid;
    const int nxt = kind == ITEM_STRESS ? ntxs[b] : (kind == ITEM_LB ? ntxl[b] : ntx[b]);
    const int ws = kind == ITEM_STRESS ? tile_width(g, 4, b) : (kind == ITEM_LB ? 32 : tile_width(g, 2, b));
    for (int yi = 0; yi < nty[b]; ++yi)
      for (int xi = 0; xi < nxt; ++xi) {
        StepItem I = blank(kind, b);
        I.x0 = ws * xi;
        I.y0 = ty * yi;
        I.z0 = zc * c;
        const int p = kind;  // ITEM_STRESS, ITEM_LB, ITEM_LC are 0, 1, 2
        if (p == 1) neighbour_waits(I, b, 0, c);
        if (p == 2) neighbour_waits(I, b, 1, c);
        if (p == 2) I.part = PL.start[b] + (c * nty[b] + yi) * ntx[b] + xi;
        if (p == 1 && stall) {
          I.wc[3] = never;
          I.wt[3] = 1;
          stall = false;
        }
        I.dc[0] = cnt(b, p, c);
        I.dc[1] = base[b] + 3 * nzc[b] + p;
        (void)G;
        it.push_back(I);
      }
  };
  for (int w = 0; w < maxz + 4; ++w)
    for (int b = 0; b < nb; ++b) {
      const int n = nzc[b], tpc = ntx[b] * nty[b], tpcs = ntxs[b] * nty[b], tpcl = ntxl[b] * nty[b],
                all = base[b] + 3 * n;
      if (w < n) tiles(ITEM_STRESS, b, chunk_of(b, w));
      if (w - 2 >= 0 && w - 2 < n) {
        tiles(ITEM_LB, b, chunk_of(b, w - 2));
        if (w - 2 == n - 1)
          for (int k = 0; k < nlk[b]; ++k) {
            StepItem I = blank(ITEM_LINKS, b);
            I.x0 = k * LINK_CHUNK;
            I.wc[0] = all + 1;
            I.wt[0] = n * tpcl;
            I.dc[0] = all + 3;
            it.push_back(I);
          }
      }
      if (w - 4 >= 0 && w - 4 < n) {
        tiles(ITEM_LC, b, chunk_of(b, w - 4));
        if (w - 4 == n - 1) {
          StepItem I = blank(ITEM_COLLOID, b);
          for (int k = 0; k < 3; ++k) {
            I.wc[k] = all + k;
            I.wt[k] = n * (k == 0 ? tpcs : (k == 1 ? tpcl : tpc));
          }
          if (nlk[b] > 0) {
            I.wc[3] = all + 3;
            I.wt[3] = nlk[b];
          }
          it.push_back(I);
        }
      }
    }
  if ((int)it.size() > g->items_cap) {
    if (g->d_items) g->mem.put(g->d_items, g->al);
    g->items_cap = (int)it.size() + 256;
    g->d_items = (StepItem*)galloc(g, sizeof(StepItem) * g->items_cap);
    if (!g->d_items) return fail(&g->err, LC_ERR_OOM, "step item list allocation failed");
  }
  if (ncnt > g->sync_cap) {
    if (g->d_sync) g->mem.put(g->d_sync, g->al);
    g->sync_cap = ncnt + 64;
    g->d_sync = (unsigned*)galloc(g, sizeof(unsigned) * g->sync_cap);
    if (!g->d_sync) return fail(&g->err, LC_ERR_OOM, "step counter allocation failed");
  }
  g->nitems = (int)it.size();
  g->nsync = ncnt;
  CK(cudaMemcpyAsync(g->d_items, it.data(), sizeof(StepItem) * it.size(), cudaMemcpyHostToDevice, g->stream),
     &g->err);
  g->step_grid = g->nsm * step_blocks_per_sm(g->prec, ty);
  return LC_OK;
}

// Polls of a dependency wait before k_step gives up (about a second);
// LCLB_SPIN_LIMIT overrides it.
int spin_limit() {
  const char* e = getenv("LCLB_SPIN_LIMIT");
  if (e && e[0]) return std::max(0, atoi(e));
  return 1 << 23;
}

cudaError_t launch_dataflow(Group* g, int commit) {
  cudaError_t e = cudaMemsetAsync(g->d_sync, 0, sizeof(unsigned) * g->nsync, g->stream);
  if (e != cudaSuccess) return e;
  return launch_step(g->prec, g->step_cfg.ty, g->d_boxes, g->d_items, g->nitems, g->step_cfg.zc, g->d_sync,
                     g->ph[2].d_part, spin_limit(), commit, g->d_err, g->step_grid, g->stream);
}

// The step kernels leave two error words in the group: d_err[0], a wait of
// k_step that gave up (the state is invalid); d_err[1], a colloid move that
// was not made because it would have touched another colloid or a wall (the
// state is valid; the first contact is in the state of its box).  Reports the
// first of them and clears both; synchronises the stream.
int check_step_err(Group* g, std::string* err) {
  int* hv = reinterpret_cast<int*>(g->h_red + 63);
  CK(cudaMemcpyAsync(hv, g->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, g->stream), err);
  CK(cudaStreamSynchronize(g->stream), err);
  if (hv[0] == 0 && hv[1] == 0) return LC_OK;
  const bool timeout = hv[0] != 0;
  CK(cudaMemsetAsync(g->d_err, 0, 2 * sizeof(int), g->stream), err);
  long long cstep = -1;
  int cbox = -1, ccol = -1, cpartner = -2;
  for (size_t b = 0; b < g->boxes.size(); ++b) {
    DevState st{};
    CK(cudaMemcpyAsync(&st, g->boxes[b]->hb.st, sizeof(st), cudaMemcpyDeviceToHost, g->stream), err);
    CK(cudaStreamSynchronize(g->stream), err);
    if (st.cstep < 0) continue;
    if (cbox < 0) {
      cbox = (int)b;
      cstep = st.cstep;
      ccol = st.ccol;
      cpartner = st.cpartner;
    }
    st.cstep = -1;
    st.err &= ~8;
    CK(cudaMemcpyAsync(g->boxes[b]->hb.st, &st, sizeof(st), cudaMemcpyHostToDevice, g->stream), err);
  }
  CK(cudaStreamSynchronize(g->stream), err);
  if (timeout) return fail(err, LC_ERR_TIMEOUT, "a dependency wait of the persistent step kernel gave up; the state is invalid");
  if (cbox < 0) return fail(err, LC_ERR_STATE, "contact flagged with no box recording it");
  char with[32];
  if (cpartner == -1) snprintf(with, sizeof(with), "a wall");
  else snprintf(with, sizeof(with), "colloid %d", cpartner);
  return fail(err, LC_ERR_OVERLAP, "step %lld: colloid %d of box %d would touch %s; it was not moved", cstep, ccol,
              cbox, with);
}

// One coupled step: fused stress + body force + collide/stream, then the Q
// update on the main stream and the link momentum exchange on the side
// stream (both read only what the fused kernel wrote), joined before the
// colloid update.
int enqueue_force_lb(Group* g) {
  if (g->variant == 1) return enqueue_split(g, FORCE_ACC);
  if (g->variant == 2) {
    CK(launch_phase(g, 4, FORCE_ACC), &g->err);
    CK(launch_phase(g, 5, 0), &g->err);
    return LC_OK;
  }
  CK(launch_phase(g, 3, FORCE_ACC), &g->err);
  return LC_OK;
}

int enqueue_step(Group* g) {
  if (g->variant == 3) {
    CK(launch_dataflow(g, 1), &g->err);
    if (g->nmob > 0)
      CK(launch_rediscretise(g->prec, g->d_boxes, (int)g->boxes.size(), g->d_mob, g->nmob, g->nsm, g->stream),
         &g->err);
    return LC_OK;
  }
  if (int rc = enqueue_force_lb(g)) return rc;
  if (g->nchunks > 0) {
    CK(cudaEventRecord(g->ev_fork, g->stream), &g->err);
    CK(cudaStreamWaitEvent(g->side, g->ev_fork, 0), &g->err);
    CK(launch_links(g->prec, g->d_boxes, g->d_chunks, g->nchunks, g->nchunks, g->side), &g->err);
    CK(cudaEventRecord(g->ev_join, g->side), &g->err);
  }
  CK(launch_phase(g, 2, LC_RESID), &g->err);
  if (g->nchunks > 0) CK(cudaStreamWaitEvent(g->stream, g->ev_join, 0), &g->err);
  CK(launch_colloid(g->d_boxes, (int)g->boxes.size(), g->stream), &g->err);
  if (g->nmob > 0)
    CK(launch_rediscretise(g->prec, g->d_boxes, (int)g->boxes.size(), g->d_mob, g->nmob, g->nsm, g->stream), &g->err);
  return LC_OK;
}

// Mobile colloid list of the group and change-list capacity of each box.
int build_mobile(Group* g) {
  std::vector<int2> mob;
  for (size_t b = 0; b < g->boxes.size(); ++b) {
    lc_lb* h = g->boxes[b];
    int need = 0;
    for (size_t c = 0; c < h->col.size(); ++c)
      if (h->col[c].mobile) {
        mob.push_back(make_int2((int)b, (int)c));
        const int e = (int)std::ceil(2.0 * h->col[c].a0) + 5;
        need += e * e * e;
      }
    if (need > h->hb.chg_cap) {
      if (h->hb.chg) g->mem.put(h->hb.chg, g->al);
      h->hb.chg = (int*)galloc(g, sizeof(int) * 2 * (size_t)need);
      if (!h->hb.chg) return fail(&h->err, LC_ERR_OOM, "change-list allocation failed");
      h->hb.chg_cap = need;
      int rc = upload_box(g, h);
      if (rc) return rc;
    }
  }
  if ((int)mob.size() > g->mob_cap) {
    if (g->d_mob) g->mem.put(g->d_mob, g->al);
    g->mob_cap = (int)mob.size() + 8;
    g->d_mob = (int2*)galloc(g, sizeof(int2) * g->mob_cap);
    if (!g->d_mob) return fail(&g->err, LC_ERR_OOM, "mobile list allocation failed");
  }
  g->nmob = (int)mob.size();
  if (!mob.empty())
    CK(cudaMemcpyAsync(g->d_mob, mob.data(), sizeof(int2) * mob.size(), cudaMemcpyHostToDevice, g->stream), &g->err);
  g->dirty = true;
  return LC_OK;
}

int capture(Group* g) {
  if (!g->dirty && g->gexec) return LC_OK;
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  if (g->graph) {
    cudaGraphDestroy(g->graph);
    g->graph = nullptr;
  }
  if (g->variant == 3)
    if (int rc = build_items(g)) return rc;
  CK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal), &g->err);
  int rc = enqueue_step(g);
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->stream, &gr);
  if (rc) {
    if (gr) cudaGraphDestroy(gr);
    return rc;
  }
  CK(e, &g->err);
  g->graph = gr;
  CK(cudaGraphInstantiate(&g->gexec, gr, 0), &g->err);
  size_t nn = 0;
  CK(cudaGraphGetNodes(gr, nullptr, &nn), &g->err);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) CK(cudaGraphGetNodes(gr, nodes.data(), &nn), &g->err);
  g->graph_kernels = 0;
  for (cudaGraphNode_t n : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(n, &t), &g->err);
    if (t == cudaGraphNodeTypeKernel) ++g->graph_kernels;
  }
  g->dirty = false;
  return LC_OK;
}

// Non-graph steps with events around each phase; mean ms per launch.
// Non-graph steps with every kernel on the main stream and events around
// each part; ms[0..4] = mean ms per step of the force + LB part, the Q
// update, the link exchange, the colloid update and the whole step; ms[5] =
// the variant, ms[6], ms[7] = the two kernels of the force + LB part (fused:
// k_flb and 0; split: k_force and k_lb, run one after the other here;
// stored: k_stress and k_lbp).
int group_profile(Group* g, int n, double* ms) {
  int rc = maybe_tune(g);
  if (rc) return rc;
  cudaEvent_t ev[6];
  for (int k = 0; k < 6; ++k) CK(cudaEventCreate(&ev[k]), &g->err);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int k1 = g->variant == 0 ? 3 : (g->variant == 1 ? 0 : 4);
  const int k2 = g->variant == 0 ? -1 : (g->variant == 1 ? 1 : 5);
  for (int s = 0; s < n; ++s) {
    CK(cudaEventRecord(ev[0], g->stream), &g->err);
    CK(launch_phase(g, k1, FORCE_ACC), &g->err);
    CK(cudaEventRecord(ev[5], g->stream), &g->err);
    if (k2 >= 0) CK(launch_phase(g, k2, 0), &g->err);
    CK(cudaEventRecord(ev[1], g->stream), &g->err);
    CK(launch_phase(g, 2, LC_RESID), &g->err);
    CK(cudaEventRecord(ev[2], g->stream), &g->err);
    CK(launch_links(g->prec, g->d_boxes, g->d_chunks, g->nchunks, g->nchunks, g->stream), &g->err);
    CK(cudaEventRecord(ev[3], g->stream), &g->err);
    CK(launch_colloid(g->d_boxes, (int)g->boxes.size(), g->stream), &g->err);
    if (g->nmob > 0)
      CK(launch_rediscretise(g->prec, g->d_boxes, (int)g->boxes.size(), g->d_mob, g->nmob, g->nsm, g->stream),
         &g->err);
    CK(cudaEventRecord(ev[4], g->stream), &g->err);
    CK(cudaEventSynchronize(ev[4]), &g->err);
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[0], ev[4]);
    acc[4] += t;
    cudaEventElapsedTime(&t, ev[0], ev[5]);
    acc[5] += t;
  }
  for (int k = 0; k < 5; ++k) ms[k] = acc[k] / n;
  if (g->variant == 3) {
    // the step as it runs: one persistent launch (whole-step time in ms[4])
    if (g->dirty && (rc = build_items(g))) return rc;
    CK(cudaEventRecord(ev[0], g->stream), &g->err);
    for (int s = 0; s < n; ++s) {
      CK(launch_dataflow(g, 1), &g->err);
      if (g->nmob > 0)
        CK(launch_rediscretise(g->prec, g->d_boxes, (int)g->boxes.size(), g->d_mob, g->nmob, g->nsm, g->stream),
           &g->err);
    }
    CK(cudaEventRecord(ev[4], g->stream), &g->err);
    CK(cudaEventSynchronize(ev[4]), &g->err);
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[0], ev[4]);
    ms[4] = t / n;
    if ((rc = check_step_err(g, &g->err))) return rc;
  }
  for (int k = 0; k < 6; ++k) cudaEventDestroy(ev[k]);
  ms[5] = g->variant;
  ms[6] = acc[5] / n;
  ms[7] = k2 >= 0 ? (acc[0] - acc[5]) / n : 0.0;
  return LC_OK;
}

int group_step(Group* g, int n) {
  if (n < 0) return fail(&g->err, LC_ERR_ARG, "negative step count");
  if (n == 0) return LC_OK;
  int rc = maybe_tune(g);
  if (rc) return rc;
  const char* env = getenv("LCLB_NO_GRAPH");
  if (env && env[0] == '1') {
    if (g->variant == 3 && g->dirty) {
      if ((rc = build_items(g))) return rc;
      g->dirty = false;
    }
    for (int s = 0; s < n; ++s)
      if ((rc = enqueue_step(g))) return rc;
    return LC_OK;
  }
  if ((rc = capture(g))) return rc;
  for (int s = 0; s < n; ++s) CK(cudaGraphLaunch(g->gexec, g->stream), &g->err);
  return LC_OK;
}

// Residual (RMS, max) of the last step of box b -> h_red[0..1] (synchronises).
int box_residual(Group* g, int b, double* rms, double* mx, long long nfluid) {
  Phase& P = g->ph[2];
  const int rec = part_records(P, 2);
  CK(launch_reduce(P.d_part, P.start[b] * rec, P.count[b] * rec, 2, 2u, g->d_red, g->stream), &g->err);
  CK(cudaMemcpyAsync(g->h_red, g->d_red, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->stream), &g->err);
  CK(cudaStreamSynchronize(g->stream), &g->err);
  *rms = nfluid > 0 ? std::sqrt(g->h_red[0] / (double)nfluid) : 0.0;
  if (int rc = check_step_err(g, &g->err)) return rc;
  *mx = g->h_red[1];
  return LC_OK;
}

int count_fluid(Group* g, lc_lb* h, long long* nf, long long* ndef, double* sums) {
  const int nb = diag_state_blocks(h->hb.N);
  int rc = ensure_scratch(g, (size_t)6 * nb);
  if (rc) return rc;
  CK(launch_diag_state(g->prec, g->d_boxes, h->index, h->hb.N, g->d_scratch, g->stream), &h->err);
  CK(launch_reduce(g->d_scratch, 0, nb, 6, 0u, g->d_red, g->stream), &h->err);
  CK(cudaMemcpyAsync(g->h_red, g->d_red, 6 * sizeof(double), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  if (sums)
    for (int k = 0; k < 4; ++k) sums[k] = g->h_red[k];
  *nf = (long long)llround(g->h_red[4]);
  if (ndef) *ndef = (long long)llround(g->h_red[5]);
  return LC_OK;
}

int rebuild_geometry(lc_lb* h) {
  Group* g = h->g;
  cudaStream_t s = g->stream;
  int rc = upload_box(g, h);
  if (rc) return rc;
  CK(launch_geometry(g->d_boxes, h->index, h->hb.N, s), &h->err);
  // boundary links, colloid by colloid, in node order
  const int nb = (h->hb.N + 255) / 256;
  if ((rc = ensure_iwork(g, (size_t)nb + 8))) return rc;
  int total = 0;
  std::vector<int> counts(h->col.size());
  for (size_t c = 0; c < h->col.size(); ++c) {
    CK(launch_link_build(g->d_boxes, h->index, h->hb.N, (int)c, g->d_iwork, total, g->d_iwork + nb, s), &h->err);
    int t = 0;
    CK(cudaMemcpyAsync(&t, g->d_iwork + nb, sizeof(int), cudaMemcpyDeviceToHost, s), &h->err);
    CK(cudaStreamSynchronize(s), &h->err);
    total = t;
  }
  if (total > h->hb.nlinks_cap) {
    if (h->hb.link_node) {
      g->mem.put(h->hb.link_node, g->al);
      g->mem.put(h->hb.link_dir, g->al);
      g->mem.put(h->hb.link_col, g->al);
    }
    const int cap = total + total / 2 + 256;
    h->hb.link_node = (int*)galloc(g, sizeof(int) * cap);
    h->hb.link_dir = (int8_t*)galloc(g, cap);
    h->hb.link_col = (int8_t*)galloc(g, cap);
    if (!h->hb.link_node || !h->hb.link_dir || !h->hb.link_col) return fail(&h->err, LC_ERR_OOM, "link allocation");
    h->hb.nlinks_cap = cap;
    if ((rc = upload_box(g, h))) return rc;
    total = 0;
    for (size_t c = 0; c < h->col.size(); ++c) {
      CK(launch_link_build(g->d_boxes, h->index, h->hb.N, (int)c, g->d_iwork, total, g->d_iwork + nb, s), &h->err);
      int t = 0;
      CK(cudaMemcpyAsync(&t, g->d_iwork + nb, sizeof(int), cudaMemcpyDeviceToHost, s), &h->err);
      CK(cudaStreamSynchronize(s), &h->err);
      total = t;
    }
  }
  CK(cudaMemcpyAsync(h->hb.nlinks, &total, sizeof(int), cudaMemcpyHostToDevice, s), &h->err);
  h->nlinks = total;
  if ((rc = build_chunks(g))) return rc;
  CK(cudaStreamSynchronize(s), &h->err);
  return LC_OK;
}

int h_check(lc_lb* h) {
  if (!h) return fail(nullptr, LC_ERR_ARG, "null handle");
  return LC_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int lc_lb_set_allocator(lc_alloc_fn alloc, lc_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(nullptr, LC_ERR_ARG, "alloc and free must both be set");
  std::lock_guard<std::mutex> lk(g_mu);
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return LC_OK;
}

const char* lc_lb_version(void) { return "lclb 0.1 (sm_103a)"; }

int lc_lb_create(const lc_grid* grid, const lc_params* params, void* stream, lc_lb** out) {
  if (!out) return fail(nullptr, LC_ERR_ARG, "null output pointer");
  *out = nullptr;
  std::string err;
  int rc = check_params(grid, params, &err);
  if (rc) return rc;
  Group* g = new_group(params->precision, stream, 1, &err);
  if (!g) return LC_ERR_OOM;
  lc_lb* h = new lc_lb();
  h->g = g;
  h->index = 0;
  h->owns_group = true;
  g->boxes.push_back(h);
  rc = make_box(g, grid, params, h);
  if (!rc) rc = rebuild_geometry(h);
  for (int k = 0; k < NPHASE && !rc; ++k) rc = build_phase(g, k);
  if (!rc) rc = build_chunks(g);
  if (rc) {
    g_err = h->err.empty() ? g->err : h->err;
    free_group(g);
    return rc;
  }
  CK(cudaStreamSynchronize(g->stream), nullptr);
  *out = h;
  return LC_OK;
}

void lc_lb_destroy(lc_lb* h) {
  if (!h || !h->owns_group) return;
  free_group(h->g);
}

int lc_lb_init_uniaxial(lc_lb* h, const double n[3], double noise_amp, uint64_t seed) {
  if (int rc = h_check(h)) return rc;
  if (!n || !(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] > 0.0)) return fail(&h->err, LC_ERR_ARG, "director must be non-zero");
  Group* g = h->g;
  const size_t N = (size_t)h->hb.N, ts = tsize(g->prec);
  CK(launch_init_q(g->prec, g->d_boxes, h->index, h->hb.N, 0, n, noise_amp, (unsigned long long)seed, g->stream),
     &h->err);
  for (int k = 0; k < 2; ++k) CK(cudaMemsetAsync(h->hb.f[k], 0, NQ * N * ts, g->stream), &h->err);
  CK(cudaMemsetAsync(h->hb.u, 0, 3 * N * ts, g->stream), &h->err);
  return write_state(g, h, 1);
}

int lc_lb_init_helix(lc_lb* h, int axis, double noise_amp, uint64_t seed) {
  if (int rc = h_check(h)) return rc;
  if (axis < 0 || axis > 2) return fail(&h->err, LC_ERR_ARG, "axis must be 0, 1 or 2");
  Group* g = h->g;
  const size_t N = (size_t)h->hb.N, ts = tsize(g->prec);
  const double n[3] = {(double)axis, 0.0, 0.0};
  CK(launch_init_q(g->prec, g->d_boxes, h->index, h->hb.N, 1, n, noise_amp, (unsigned long long)seed, g->stream),
     &h->err);
  for (int k = 0; k < 2; ++k) CK(cudaMemsetAsync(h->hb.f[k], 0, NQ * N * ts, g->stream), &h->err);
  CK(cudaMemsetAsync(h->hb.u, 0, 3 * N * ts, g->stream), &h->err);
  return write_state(g, h, 1);
}

int lc_lb_set_fields(lc_lb* h, int which, const void* src, size_t bytes, int src_is_device) {
  if (int rc = h_check(h)) return rc;
  Group* g = h->g;
  const size_t N = (size_t)h->hb.N;
  size_t nc = which == LC_Q ? 5 : (which == LC_F_PRE ? NQ : 0);
  if (!nc) return fail(&h->err, LC_ERR_ARG, "only LC_Q and LC_F_PRE can be set");
  if (!src || bytes != nc * N * sizeof(double)) return fail(&h->err, LC_ERR_ARG, "expected %zu bytes", nc * N * 8);
  int rc = ensure_scratch(g, nc * N);
  if (rc) return rc;
  CK(cudaMemcpyAsync(g->d_scratch, src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     g->stream),
     &h->err);
  if (which == LC_F_PRE) {
    // the pre-collision state goes into the current buffer and is read in place
    DevState st{};
    CK(cudaMemcpyAsync(&st, h->hb.st, sizeof(st), cudaMemcpyDeviceToHost, g->stream), &h->err);
    CK(cudaStreamSynchronize(g->stream), &h->err);
    CK(launch_set_field(g->prec, g->d_boxes, h->index, h->hb.N, 1, g->d_scratch, g->stream), &h->err);
    st.pre_valid = 1;
    CK(cudaMemcpyAsync(h->hb.st, &st, sizeof(st), cudaMemcpyHostToDevice, g->stream), &h->err);
  } else {
    CK(launch_set_field(g->prec, g->d_boxes, h->index, h->hb.N, 0, g->d_scratch, g->stream), &h->err);
  }
  CK(cudaStreamSynchronize(g->stream), &h->err);
  return LC_OK;
}

int lc_lb_add_colloid(lc_lb* h, const double X[3], double a0, int anchoring, double w, int mobile,
                      const double F_ext[3], int* id_out) {
  if (int rc = h_check(h)) return rc;
  if (!X || !(a0 > 0.0)) return fail(&h->err, LC_ERR_ARG, "bad colloid position or radius");
  if ((int)h->col.size() >= MAXCOL) return fail(&h->err, LC_ERR_ARG, "too many colloids (max %d)", MAXCOL);
  if (anchoring != LC_NORMAL && anchoring != LC_PLANAR) return fail(&h->err, LC_ERR_ARG, "unknown anchoring");
  if (h->grid.wall_z && (X[2] - a0 < -0.5 || X[2] + a0 > h->grid.nz - 0.5))
    return fail(&h->err, LC_ERR_OVERLAP, "colloid crosses a wall");
  Group* g = h->g;
  if (!h->col.empty()) {
    // contact test against the current positions (mobile colloids move on the device)
    std::vector<DevColloid> cur(h->col.size());
    CK(cudaMemcpyAsync(cur.data(), h->hb.col, sizeof(DevColloid) * cur.size(), cudaMemcpyDeviceToHost, g->stream),
       &h->err);
    CK(cudaStreamSynchronize(g->stream), &h->err);
    const int L[3] = {h->grid.nx, h->grid.ny, h->grid.nz};
    for (size_t d = 0; d < cur.size(); ++d) {
      double r2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        double r = X[a] - cur[d].X[a];
        if (a < 2 || !h->grid.wall_z) {
          if (r >= 0.5 * L[a]) r -= L[a];
          else if (r < -0.5 * L[a]) r += L[a];
        }
        r2 += r * r;
      }
      const double s = a0 + cur[d].a0;
      if (r2 < s * s) return fail(&h->err, LC_ERR_OVERLAP, "colloid touches colloid %d", (int)d);
    }
  }
  DevColloid C;
  memset(&C, 0, sizeof(C));
  for (int a = 0; a < 3; ++a) {
    C.X[a] = C.Xb[a] = X[a];
    C.Fext[a] = F_ext ? F_ext[a] : 0.0;
  }
  C.a0 = a0;
  C.w = w;
  C.strong = (!(w > 0.0) || std::isinf(w)) ? 1 : 0;
  C.wfac = C.strong ? 1.0 : w / (h->hb.p.K + w);
  C.anchoring = anchoring;
  C.mobile = mobile ? 1 : 0;
  C.M = h->params.rho0 * 4.0 / 3.0 * M_PI * a0 * a0 * a0;
  C.I = 0.4 * C.M * a0 * a0;
  const int id = (int)h->col.size();
  CK(cudaMemcpyAsync(h->hb.col + id, &C, sizeof(C), cudaMemcpyHostToDevice, g->stream), &h->err);
  h->col.push_back(C);
  h->hb.ncol = (int)h->col.size();
  h->hb.nmobile += C.mobile;
  int rc = rebuild_geometry(h);
  if (rc) return rc;
  DevState st{};
  CK(cudaMemcpyAsync(&st, h->hb.st, sizeof(st), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  if (st.err & 4) {
    h->col.pop_back();
    h->hb.ncol = (int)h->col.size();
    h->hb.nmobile -= C.mobile;
    st.err &= ~4;
    CK(cudaMemcpyAsync(h->hb.st, &st, sizeof(st), cudaMemcpyHostToDevice, g->stream), &h->err);
    rc = rebuild_geometry(h);
    if (rc) return rc;
    return fail(&h->err, LC_ERR_OVERLAP, "colloid overlaps another colloid");
  }
  if (C.mobile && (rc = build_mobile(g))) return rc;
  if (id_out) *id_out = id;
  return LC_OK;
}

static int colloid_rmw(lc_lb* h, int id, const double* V, const double* W, const double* Fext,
                       const double* Text = nullptr) {
  if (int rc = h_check(h)) return rc;
  if (id < 0 || id >= (int)h->col.size()) return fail(&h->err, LC_ERR_ARG, "no colloid %d", id);
  Group* g = h->g;
  DevColloid C;
  CK(cudaMemcpyAsync(&C, h->hb.col + id, sizeof(C), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  for (int a = 0; a < 3; ++a) {
    if (V) C.V[a] = C.Vb[a] = V[a];
    if (W) C.W[a] = C.Wb[a] = W[a];
    if (Fext) C.Fext[a] = Fext[a];
    if (Text) C.Text[a] = Text[a];
  }
  CK(cudaMemcpyAsync(h->hb.col + id, &C, sizeof(C), cudaMemcpyHostToDevice, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  return LC_OK;
}

int lc_lb_set_colloid_velocity(lc_lb* h, int id, const double V[3], const double W[3]) {
  return colloid_rmw(h, id, V, W, nullptr);
}

int lc_lb_set_colloid_force(lc_lb* h, int id, const double F_ext[3]) { return colloid_rmw(h, id, nullptr, nullptr, F_ext); }

int lc_lb_set_colloid_torque(lc_lb* h, int id, const double T_ext[3]) {
  if (!T_ext) return fail(h ? &h->err : nullptr, LC_ERR_ARG, "null torque");
  return colloid_rmw(h, id, nullptr, nullptr, nullptr, T_ext);
}

int lc_lb_step(lc_lb* h, int nsteps) {
  if (int rc = h_check(h)) return rc;
  if (!h->owns_group) return fail(&h->err, LC_ERR_STATE, "box of a batch: step the batch");
  int rc = group_step(h->g, nsteps);
  if (rc) h->err = h->g->err;
  return rc;
}

int lc_lb_synchronize(lc_lb* h) {
  if (int rc = h_check(h)) return rc;
  CK(cudaStreamSynchronize(h->g->stream), &h->err);
  return check_step_err(h->g, &h->err);
}

int lc_lb_relax(lc_lb* h, double tol, long long max_steps, int check_every, long long* steps_out, double* resid_out) {
  if (int rc = h_check(h)) return rc;
  if (!h->owns_group) return fail(&h->err, LC_ERR_STATE, "box of a batch: relax the batch");
  if (check_every < 1 || max_steps < 0) return fail(&h->err, LC_ERR_ARG, "bad relax arguments");
  Group* g = h->g;
  long long nf = 0;
  int rc = count_fluid(g, h, &nf, nullptr, nullptr);
  if (rc) return rc;
  long long done = 0;
  double rms = INFINITY, mx = 0.0;
  while (done < max_steps) {
    const int n = (int)std::min<long long>(check_every, max_steps - done);
    if ((rc = group_step(g, n))) {
      h->err = g->err;
      return rc;
    }
    done += n;
    if ((rc = box_residual(g, h->index, &rms, &mx, nf))) return rc;
    if (!std::isfinite(rms)) {
      if (steps_out) *steps_out = done;
      if (resid_out) *resid_out = rms;
      return fail(&h->err, LC_ERR_NONFINITE, "residual is not finite after %lld steps", done);
    }
    if (rms <= tol) break;
  }
  if (steps_out) *steps_out = done;
  if (resid_out) *resid_out = rms;
  return LC_OK;
}

int lc_lb_get_fields(lc_lb* h, int which, void* dst, size_t bytes, int dst_is_device) {
  if (int rc = h_check(h)) return rc;
  Group* g = h->g;
  const size_t N = (size_t)h->hb.N;
  size_t nc = 0;
  switch (which) {
    case LC_Q: nc = 5; break;
    case LC_U: nc = 3; break;
    case LC_RHO: nc = 1; break;
    case LC_F_PRE: nc = NQ; break;
    case LC_FORCE: nc = 3; break;
    case LC_SOLID: nc = 1; break;
    default: return fail(&h->err, LC_ERR_ARG, "unknown field %d", which);
  }
  if (!dst || bytes < nc * N * sizeof(double)) return fail(&h->err, LC_ERR_ARG, "destination too small");
  int rc = ensure_scratch(g, nc * N);
  if (rc) return rc;
  if ((which == LC_U || which == LC_FORCE) && h->hb.p.lc_on) {
    // body force of the current Q (no colloid accumulation)
    CK(launch_phase(g, 0, 0, h->index), &h->err);
  }
  CK(launch_export(g->prec, g->d_boxes, h->index, h->hb.N, which, g->d_scratch, g->stream), &h->err);
  CK(cudaMemcpyAsync(dst, g->d_scratch, nc * N * sizeof(double),
                     dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream),
     &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  return check_step_err(g, &h->err);
}

int lc_lb_get_colloid(lc_lb* h, int id, double out[27]) {
  if (int rc = h_check(h)) return rc;
  if (id < 0 || id >= (int)h->col.size() || !out) return fail(&h->err, LC_ERR_ARG, "no colloid %d", id);
  DevColloid C;
  CK(cudaMemcpyAsync(&C, h->hb.col + id, sizeof(C), cudaMemcpyDeviceToHost, h->g->stream), &h->err);
  CK(cudaStreamSynchronize(h->g->stream), &h->err);
  if (int rc = check_step_err(h->g, &h->err)) return rc;
  const double* src[9] = {C.X, C.V, C.W, C.Fh, C.Th, C.Flc, C.Tlc, C.imp, C.aimp};
  for (int k = 0; k < 9; ++k)
    for (int a = 0; a < 3; ++a) out[3 * k + a] = src[k][a];
  return LC_OK;
}

int lc_lb_get_forces(lc_lb* h, int id, double F[3], double T[3], double V[3], double W[3], double X[3]) {
  double r[27];
  int rc = lc_lb_get_colloid(h, id, r);
  if (rc) return rc;
  for (int a = 0; a < 3; ++a) {
    if (F) F[a] = r[9 + a] + r[15 + a];
    if (T) T[a] = r[12 + a] + r[18 + a];
    if (V) V[a] = r[3 + a];
    if (W) W[a] = r[6 + a];
    if (X) X[a] = r[a];
  }
  return LC_OK;
}

int lc_lb_get_links(lc_lb* h, int32_t* node, int8_t* dir, int16_t* colloid, size_t cap, size_t* n_out) {
  if (int rc = h_check(h)) return rc;
  Group* g = h->g;
  int n = 0;
  CK(cudaMemcpyAsync(&n, h->hb.nlinks, sizeof(int), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  if (n_out) *n_out = (size_t)n;
  const size_t k = std::min(cap, (size_t)n);
  if (k == 0) return LC_OK;
  // the device list is in node order after a full build and unordered after a
  // re-discretisation: return it sorted by (colloid, node, direction)
  std::vector<int> nd((size_t)n);
  std::vector<int8_t> dr((size_t)n), c8((size_t)n);
  CK(cudaMemcpyAsync(nd.data(), h->hb.link_node, sizeof(int) * n, cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaMemcpyAsync(dr.data(), h->hb.link_dir, n, cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaMemcpyAsync(c8.data(), h->hb.link_col, n, cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  std::vector<size_t> ord((size_t)n);
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
    if (c8[a] != c8[b]) return c8[a] < c8[b];
    if (nd[a] != nd[b]) return nd[a] < nd[b];
    return dr[a] < dr[b];
  });
  for (size_t i = 0; i < k; ++i) {
    if (node) node[i] = nd[ord[i]];
    if (dir) dir[i] = dr[ord[i]];
    if (colloid) colloid[i] = c8[ord[i]];
  }
  return LC_OK;
}

// Labels the defect nodes of box h (see lc_lb_defects): parent[i] = the
// smallest node index of i's component, or -1, in h->def; the components
// numbered in root order.  *ncomp receives their number.
static int defects_label(lc_lb* h, double thr, int* ncomp) {
  if (!(thr > 0.0) || !std::isfinite(thr)) return fail(&h->err, LC_ERR_ARG, "defect threshold must be positive");
  Group* g = h->g;
  const int N = h->hb.N;
  const int nb = defect_blocks(N);
  const size_t need = (size_t)3 * N + nb + 2;
  if (h->def_cap < need) {
    if (h->def) g->mem.put(h->def, g->al);
    h->def = (int*)galloc(g, sizeof(int) * need);
    h->def_cap = h->def ? need : 0;
    if (!h->def) return fail(&h->err, LC_ERR_OOM, "defect label allocation failed");
  }
  int* parent = h->def;
  int* comp = parent + N;
  int* list = comp + N;
  int* blockcnt = list + N;
  int* total = blockcnt + nb;
  int* errf = total + 1;
  CK(cudaMemsetAsync(errf, 0, sizeof(int), g->stream), &h->err);
  CK(launch_defects_label(g->prec, g->d_boxes, h->index, N, thr, parent, comp, list, blockcnt, total, errf, g->stream),
     &h->err);
  int hv[2] = {0, 0};
  CK(cudaMemcpyAsync(hv, total, sizeof(hv), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  if (hv[1]) return fail(&h->err, LC_ERR_TIMEOUT, "defect labelling: a bounded find/union loop gave up");
  *ncomp = hv[0];
  return LC_OK;
}

int lc_lb_defects(lc_lb* h, double thr, size_t cap, long long* n_defect, long long* n_comp, long long* root,
                  long long* size, double* centroid, double* gyration) {
  if (int rc = h_check(h)) return rc;
  int nc = 0;
  if (int rc = defects_label(h, thr, &nc)) return rc;
  Group* g = h->g;
  const int N = h->hb.N;
  std::vector<int> hl((size_t)nc), hs((size_t)nc);
  std::vector<double> hc((size_t)3 * nc), hg((size_t)6 * nc);
  if (nc > 0) {
    const size_t ib = ((sizeof(int) * (size_t)nc + 15) / 16) * 16;
    char* tmp = (char*)galloc(g, ib + sizeof(double) * 15 * (size_t)nc);
    if (!tmp) return fail(&h->err, LC_ERR_OOM, "defect statistics allocation failed");
    int* dsz = (int*)tmp;
    double* circ = (double*)(tmp + ib);
    double* cen = circ + 6 * (size_t)nc;
    double* gyr = cen + 3 * (size_t)nc;
    int rc = LC_OK;
    if (cudaMemsetAsync(tmp, 0, ib + sizeof(double) * 15 * (size_t)nc, g->stream) != cudaSuccess ||
        launch_defects_stats(g->d_boxes, h->index, N, nc, h->def, h->def + N, dsz, circ, cen, gyr, g->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(hl.data(), h->def + 2 * (size_t)N, sizeof(int) * nc, cudaMemcpyDeviceToHost, g->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(hs.data(), dsz, sizeof(int) * nc, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(hc.data(), cen, sizeof(double) * 3 * nc, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(hg.data(), gyr, sizeof(double) * 6 * nc, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
      rc = fail(&h->err, LC_ERR_CUDA, "defect statistics: %s", cudaGetErrorString(cudaGetLastError()));
    g->mem.put(tmp, g->al);
    if (rc) return rc;
  }
  long long nd = 0;
  for (int v : hs) nd += v;
  if (n_defect) *n_defect = nd;
  if (n_comp) *n_comp = nc;
  const size_t k = std::min(cap, (size_t)nc);
  for (size_t c = 0; c < k; ++c) {
    if (root) root[c] = hl[c];
    if (size) size[c] = hs[c];
    for (int a = 0; a < 3 && centroid; ++a) centroid[3 * c + a] = hc[3 * c + a];
    for (int a = 0; a < 6 && gyration; ++a) gyration[6 * c + a] = hg[6 * c + a];
  }
  return LC_OK;
}

int lc_lb_defect_labels(lc_lb* h, double thr, int32_t* labels, size_t n, int dst_is_device) {
  if (int rc = h_check(h)) return rc;
  if (!labels || n < (size_t)h->hb.N) return fail(&h->err, LC_ERR_ARG, "labels needs N = %d entries", h->hb.N);
  int nc = 0;
  if (int rc = defects_label(h, thr, &nc)) return rc;
  Group* g = h->g;
  CK(cudaMemcpyAsync(labels, h->def, sizeof(int32_t) * h->hb.N,
                     dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream),
     &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  return LC_OK;
}

int lc_lb_diagnostics(lc_lb* h, lc_diag* out) {
  if (int rc = h_check(h)) return rc;
  if (!out) return fail(&h->err, LC_ERR_ARG, "null output");
  Group* g = h->g;
  memset(out, 0, sizeof(*out));
  long long nf = 0, nd = 0;
  double sums[4];
  int rc = count_fluid(g, h, &nf, &nd, sums);
  if (rc) return rc;
  if ((rc = check_step_err(g, &h->err))) return rc;
  out->n_fluid = nf;
  out->n_defect = nd;
  out->mass = (double)nf * h->hb.p.rho0 + sums[0];
  for (int a = 0; a < 3; ++a) out->momentum[a] = sums[1 + a];
  if (h->hb.p.lc_on) {
    CK(launch_phase(g, 0, FORCE_FE, h->index), &h->err);
    Phase& P = g->ph[0];
    CK(launch_reduce(P.d_part, P.start[h->index], P.count[h->index], 1, 0u, g->d_red, g->stream), &h->err);
    CK(cudaMemcpyAsync(g->h_red, g->d_red, sizeof(double), cudaMemcpyDeviceToHost, g->stream), &h->err);
    CK(cudaStreamSynchronize(g->stream), &h->err);
    out->free_energy = g->h_red[0];
    double rms = 0, mx = 0;
    if ((rc = box_residual(g, h->index, &rms, &mx, nf))) return rc;
    out->resid_rms = rms;
    out->resid_max = mx;
  }
  DevState st{};
  CK(cudaMemcpyAsync(&st, h->hb.st, sizeof(st), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  out->step = st.step;
  if (!std::isfinite(out->mass) || !std::isfinite(out->free_energy))
    return fail(&h->err, LC_ERR_NONFINITE, "non-finite diagnostics");
  return LC_OK;
}

int lc_lb_profile_detail(lc_lb* h, int nsteps, double ms_out[8]) {
  if (int rc = h_check(h)) return rc;
  if (!h->owns_group) return fail(&h->err, LC_ERR_STATE, "box of a batch: profile the batch");
  if (nsteps < 1 || !ms_out) return fail(&h->err, LC_ERR_ARG, "bad profile arguments");
  int rc = group_profile(h->g, nsteps, ms_out);
  if (rc) h->err = h->g->err;
  return rc;
}

int lc_lb_profile(lc_lb* h, int nsteps, double ms_out[5]) {
  double ms[8];
  int rc = lc_lb_profile_detail(h, nsteps, ms_out ? ms : nullptr);
  if (!rc)
    for (int k = 0; k < 5; ++k) ms_out[k] = ms[k];
  return rc;
}

int lc_lb_step_launches(lc_lb* h, int* n_out) {
  if (int rc = h_check(h)) return rc;
  if (!n_out) return fail(&h->err, LC_ERR_ARG, "null output");
  Group* g = h->g;
  int rc = maybe_tune(g);
  if (!rc) rc = capture(g);
  if (rc) {
    h->err = g->err;
    return rc;
  }
  *n_out = g->graph_kernels;
  return LC_OK;
}

int lc_lb_batch_step_launches(lc_lb_batch* b, int* n_out) {
  if (!b || !n_out) return fail(b ? &b->err : nullptr, LC_ERR_ARG, "bad arguments");
  int rc = maybe_tune(b->g);
  if (!rc) rc = capture(b->g);
  if (rc) {
    b->err = b->g->err;
    return rc;
  }
  *n_out = b->g->graph_kernels;
  return LC_OK;
}

int lc_lb_batch_profile_detail(lc_lb_batch* b, int nsteps, double ms_out[8]) {
  if (!b || nsteps < 1 || !ms_out) return fail(b ? &b->err : nullptr, LC_ERR_ARG, "bad profile arguments");
  int rc = group_profile(b->g, nsteps, ms_out);
  if (rc) b->err = b->g->err;
  return rc;
}

int lc_lb_batch_profile(lc_lb_batch* b, int nsteps, double ms_out[5]) {
  double ms[8];
  int rc = lc_lb_batch_profile_detail(b, nsteps, ms_out ? ms : nullptr);
  if (!rc)
    for (int k = 0; k < 5; ++k) ms_out[k] = ms[k];
  return rc;
}

}  // extern "C"

// ---- diagnostics without allocation ------------------------------------------
// Scratch of lc_lb_diagnostics_noalloc: one record of 6 doubles per block of
// 256 nodes for up to 8192 blocks (2,097,152 nodes), then 8 doubles for the
// reduced values: 384 KiB + 64 B on every device that loads the library.
namespace {
constexpr int NOALLOC_MAX_BLOCKS = 8192;
constexpr int NOALLOC_OUT = NOALLOC_MAX_BLOCKS * 6;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[128] = {nullptr};
}  // namespace
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_BLOCKS * 6 + 8];

// Device address of the scratch on the current device, looked up once per
// device (the host symbol is only a stand-in, not a device address) in the
// device's primary context.  The current device must be the group's.
static int noalloc_scratch(const Group* g, double** out, std::string* err) {
  int dev = 0;
  CK(cudaGetDevice(&dev), err);
  if (dev != g->dev)
    return fail(err, LC_ERR_ARG, "current device %d is not the handle's device %d", dev, g->dev);
  if (dev < 0 || dev >= 128) return fail(err, LC_ERR_ARG, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(err, LC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return LC_OK;
}

extern "C" {

int lc_lb_diagnostics_noalloc(lc_lb* h, lc_diag* out) {
  if (int rc = h_check(h)) return rc;
  if (!out) return fail(&h->err, LC_ERR_ARG, "null output");
  const int nb = diag_state_blocks(h->hb.N);
  if (nb > NOALLOC_MAX_BLOCKS)
    return fail(&h->err, LC_ERR_ARG,
                "box of %d nodes exceeds the %d-node limit of the allocation-free diagnostics", h->hb.N,
                NOALLOC_MAX_BLOCKS * 256);
  double* scr = nullptr;
  int rc = noalloc_scratch(h->g, &scr, &h->err);
  if (rc) return rc;
  Group* g = h->g;
  CK(launch_diag_state(g->prec, g->d_boxes, h->index, h->hb.N, scr, g->stream), &h->err);
  CK(launch_reduce(scr, 0, nb, 6, 0u, scr + NOALLOC_OUT, g->stream), &h->err);
  double r[6];
  DevState st{};
  CK(cudaMemcpyAsync(r, scr + NOALLOC_OUT, sizeof(r), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaMemcpyAsync(&st, h->hb.st, sizeof(st), cudaMemcpyDeviceToHost, g->stream), &h->err);
  CK(cudaStreamSynchronize(g->stream), &h->err);
  memset(out, 0, sizeof(*out));
  out->n_fluid = (long long)llround(r[4]);
  out->n_defect = (long long)llround(r[5]);
  out->mass = (double)out->n_fluid * h->hb.p.rho0 + r[0];
  for (int a = 0; a < 3; ++a) out->momentum[a] = r[1 + a];
  out->step = st.step;
  if (!std::isfinite(out->mass)) return fail(&h->err, LC_ERR_NONFINITE, "non-finite diagnostics");
  return LC_OK;
}

const char* lc_lb_last_error(const lc_lb* h) {
  if (!h) return g_err.c_str();
  if (!h->err.empty()) return h->err.c_str();
  return h->g ? h->g->err.c_str() : "";
}

// ---- batch ------------------------------------------------------------------
int lc_lb_batch_create(int n, const lc_grid* grids, const lc_params* params, void* stream, lc_lb_batch** out) {
  if (!out || n < 1 || !grids || !params) return fail(nullptr, LC_ERR_ARG, "bad batch arguments");
  *out = nullptr;
  std::string err;
  for (int i = 0; i < n; ++i) {
    int rc = check_params(grids + i, params + i, &err);
    if (rc) return rc;
    if (params[i].precision != params[0].precision) return fail(nullptr, LC_ERR_ARG, "mixed precision in a batch");
  }
  Group* g = new_group(params[0].precision, stream, n, &err);
  if (!g) return LC_ERR_OOM;
  int rc = LC_OK;
  for (int i = 0; i < n && !rc; ++i) {
    lc_lb* h = new lc_lb();
    h->g = g;
    h->index = i;
    g->boxes.push_back(h);
    rc = make_box(g, grids + i, params + i, h);
    if (!rc) rc = rebuild_geometry(h);
    if (rc) g_err = h->err;
  }
  for (int k = 0; k < NPHASE && !rc; ++k) rc = build_phase(g, k);
  if (!rc) rc = build_chunks(g);
  if (rc) {
    free_group(g);
    return rc;
  }
  CK(cudaStreamSynchronize(g->stream), nullptr);
  lc_lb_batch* b = new lc_lb_batch();
  b->g = g;
  *out = b;
  return LC_OK;
}

void lc_lb_batch_destroy(lc_lb_batch* b) {
  if (!b) return;
  free_group(b->g);
  delete b;
}

int lc_lb_batch_box(lc_lb_batch* b, int i, lc_lb** box) {
  if (!b || !box || i < 0 || i >= (int)b->g->boxes.size()) return fail(b ? &b->err : nullptr, LC_ERR_ARG, "no box %d", i);
  *box = b->g->boxes[i];
  return LC_OK;
}

int lc_lb_batch_step(lc_lb_batch* b, int nsteps) {
  if (!b) return fail(nullptr, LC_ERR_ARG, "null batch");
  int rc = group_step(b->g, nsteps);
  if (rc) b->err = b->g->err;
  return rc;
}

int lc_lb_batch_relax(lc_lb_batch* b, double tol, long long max_steps, int check_every, long long* steps_out,
                      double* resid_out) {
  if (!b || check_every < 1 || max_steps < 0) return fail(b ? &b->err : nullptr, LC_ERR_ARG, "bad relax arguments");
  Group* g = b->g;
  const int n = (int)g->boxes.size();
  std::vector<long long> nf(n);
  for (int i = 0; i < n; ++i) {
    int rc = count_fluid(g, g->boxes[i], &nf[i], nullptr, nullptr);
    if (rc) return rc;
  }
  std::vector<double> r(n, INFINITY);
  long long done = 0;
  while (done < max_steps) {
    const int k = (int)std::min<long long>(check_every, max_steps - done);
    int rc = group_step(g, k);
    if (rc) {
      b->err = g->err;
      return rc;
    }
    done += k;
    bool ok = true;
    for (int i = 0; i < n; ++i) {
      double mx;
      if ((rc = box_residual(g, i, &r[i], &mx, nf[i]))) return rc;
      if (!std::isfinite(r[i])) return fail(&b->err, LC_ERR_NONFINITE, "box %d residual not finite", i);
      ok = ok && r[i] <= tol;
    }
    if (ok) break;
  }
  if (steps_out) *steps_out = done;
  if (resid_out)
    for (int i = 0; i < n; ++i) resid_out[i] = r[i];
  return LC_OK;
}

const char* lc_lb_batch_last_error(const lc_lb_batch* b) {
  if (!b) return g_err.c_str();
  return b->err.empty() ? b->g->err.c_str() : b->err.c_str();
}

int lc_lb_autotune(const lc_grid* grid, int precision, void* stream, char* out_desc, size_t desc_len) {
  lc_params p;
  memset(&p, 0, sizeof(p));
  p.rho0 = 1.0; p.tau = 2.5; p.A0 = 0.01; p.gamma = 3.0; p.K = 0.01; p.q0 = 0.0; p.xi = 0.7; p.Gamma = 0.5;
  p.precision = precision; p.lc_enabled = 1; p.flow_enabled = 1;
  lc_lb* h = nullptr;
  int rc = lc_lb_create(grid, &p, stream, &h);
  if (rc) return rc;
  const double n[3] = {0.0, 0.0, 1.0};
  lc_lb_init_uniaxial(h, n, 1e-3, 1);
  std::string desc;
  rc = autotune_group(h->g, &desc);
  if (out_desc && desc_len) snprintf(out_desc, desc_len, "%s", desc.c_str());
  if (rc) g_err = h->g->err;
  lc_lb_destroy(h);
  return rc;
}

}  // extern "C"
