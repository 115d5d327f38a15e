// af_batch.cu -- the batch ABI of include/af.h: an ensemble of independent
// grids of uneven sizes advanced by batched kernels, each instance with its
// own device-side time step, whole runs captured in one CUDA graph.
//
// Each instance is a full single-grid handle (af_ctx) for its storage and
// transfers.  The batch adds, in device memory, one control block per
// instance (time, end time, dt and the dt/dx ratios, which of its two t^n
// buffers is current, status, counters, wave speed), the per-instance
// kernel arguments for both buffer assignments, the TMA descriptors for the
// chosen point-value tile height, and flat tile lists (instance, i0, j0)
// that the batched kernels walk with one block per tile.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "../../include/af.h"
#include "af_ctx.h"
#include "af_kernels.h"

using namespace af;

namespace {

constexpr int GRAPH_CHUNK = 256;  // steps per captured graph
const int TILE_HEIGHTS[3] = {4, 8, 16};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int steps = 0;
  double *hist = nullptr;
  int hist_steps = 0;
};

}  // namespace

struct af_batch {
  int n = 0;
  int device = 0;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  std::vector<af_ctx *> inst;
  int tile_h = 8;
  std::vector<BatchCtl> ctl_h;  // host mirror, current after sync_ctl
  std::vector<char> has_state, speed_ok, stopped;
  BatchCtl *d_ctl = nullptr;
  PointValueArgs *d_pv = nullptr;  // [n][2]
  FluxArgs *d_fx = nullptr;        // [n][2]
  TileMaps *d_maps = nullptr;      // [n][2]
  Grid *d_grids = nullptr;
  float **d_arrays = nullptr;      // [n][2][5]
  int4 *d_pv_tiles = nullptr, *d_fx_tiles = nullptr;
  int n_pv_tiles = 0, n_fx_tiles = 0, pv_tiles_h = 0;
  int n_fx_plain = -1;  // flux tiles of instances without the flux limiter (listed first)
  int4 *d_ghost_chunks = nullptr;  // (instance, array, first entry) per ghost-fill block
  int n_ghost_chunks = 0;
  int4 *d_theta_tiles = nullptr;   // (instance, a0, b0): shock-indicator tiles of the blending instances
  int n_theta_tiles = 0, theta_tiles_cap = 0;
  bool maps_ok = false;
  bool timed_out = false;  // an instance reported AF_ST_TIMEOUT: no further runs
  std::vector<GraphEntry> graphs;
  bool any_limiter = false;  // some instance has the flux limiter on
  bool any_blend = false;    // some instance has the Sec. 3.4 blend on
  float **d_theta = nullptr; // [n][2] blend weight planes (NULL: off)
  bool sampling = false;  // training-set sampler between point values and fluxes
  SampleBatch sampler;
};

namespace {

int bfail(int code, const char *msg) { return set_error(code, msg); }
int bcuda(cudaError_t e, const char *where) {
  char m[400];
  std::snprintf(m, sizeof(m), "%s: %s", where, cudaGetErrorString(e));
  return set_error(AF_ERR_CUDA, m);
}
#define BCK(call, where)                               \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return bcuda(e_, where);    \
  } while (0)

struct Dev {
  int old = -1;
  explicit Dev(int d) {
    if (cudaGetDevice(&old) == cudaSuccess && old != d) cudaSetDevice(d);
    else old = -1;
  }
  ~Dev() {
    if (old >= 0) cudaSetDevice(old);
  }
};

void drop_graphs(af_batch *b) {
  for (auto &e : b->graphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  b->graphs.clear();
}

// device control blocks -> host mirror; instance handles follow the buffer
// that now holds each instance's t^n
int sync_ctl(af_batch *b) {
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  BCK(cudaMemcpy(b->ctl_h.data(), b->d_ctl, sizeof(BatchCtl) * b->n, cudaMemcpyDeviceToHost), "batch: ctl");
  for (int k = 0; k < b->n; k++) {
    af_ctx *h = b->inst[k];
    const BatchCtl &c = b->ctl_h[k];
    h->tmap_cur = c.cur;
    h->lev[0] = h->tbuf[c.cur];
    h->lev[2] = h->tbuf[c.cur ^ 1];
    h->speed_valid = false;
    if (!c.active && (c.status & ST_STOPPED)) b->stopped[k] = 1;
    if (c.status & ST_TIMEOUT) b->timed_out = true;
  }
  return AF_OK;
}

int put_ctl(af_batch *b) {
  BCK(cudaMemcpyAsync(b->d_ctl, b->ctl_h.data(), sizeof(BatchCtl) * b->n, cudaMemcpyHostToDevice, b->stream),
      "batch: ctl");
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  return AF_OK;
}

// kernel arguments of every instance for both buffer assignments
int upload_args(af_batch *b) {
  std::vector<PointValueArgs> pv(2 * b->n);
  std::vector<FluxArgs> fx(2 * b->n);
  std::vector<float *> arrays(10 * (size_t)b->n);
  bool any_lim = false, any_blend = false;
  std::vector<float *> theta(2 * (size_t)b->n);
  for (int k = 0; k < b->n; k++) {
    af_ctx *h = b->inst[k];
    BatchCtl *c = b->d_ctl + k;
    for (int q = 0; q < 2; q++) {
      pv[2 * k + q] = pointvalue_args(h->g, h->tbuf[q], h->hi, h->lev[1], h->tbuf[q ^ 1], h->opt, &c->status,
                                      c->counters);
      if (h->opt.shock_blend) {
        pv[2 * k + q].theta[0] = h->shock_theta;
        pv[2 * k + q].theta[1] = h->shock_theta + h->g.plane;
      }
      fx[2 * k + q] = flux_args(h->g, h->tbuf[q], h->lev[1], h->tbuf[q ^ 1], h->hi, h->lo, &c->status, &c->speed,
                                &c->speed_bad);
      fx[2 * k + q].flux_limiter = h->opt.flux_limiter;
      if (h->opt.flux_limiter) fx[2 * k + q].q0 = h->q0;
      if (h->opt.flux_limiter) any_lim = true;
      float **a = &arrays[(2 * k + q) * 5];
      a[0] = h->hi;
      a[1] = h->lo;
      a[2] = h->tbuf[q].k[VTX];
      a[3] = h->tbuf[q].k[XE];
      a[4] = h->tbuf[q].k[YE];
    }
    theta[2 * k] = h->opt.shock_blend ? h->shock_theta : nullptr;
    theta[2 * k + 1] = h->opt.shock_blend ? h->shock_theta + h->g.plane : nullptr;
    if (h->opt.shock_blend) any_blend = true;
  }
  BCK(cudaMemcpy(b->d_pv, pv.data(), sizeof(PointValueArgs) * pv.size(), cudaMemcpyHostToDevice), "batch: args");
  BCK(cudaMemcpy(b->d_fx, fx.data(), sizeof(FluxArgs) * fx.size(), cudaMemcpyHostToDevice), "batch: args");
  BCK(cudaMemcpy(b->d_arrays, arrays.data(), sizeof(float *) * arrays.size(), cudaMemcpyHostToDevice),
      "batch: args");
  BCK(cudaMemcpy(b->d_theta, theta.data(), sizeof(float *) * theta.size(), cudaMemcpyHostToDevice),
      "batch: args");
  // flux tiles: instances without the flux limiter first (plain kernel), then
  // the limiting ones (limited kernel)
  std::vector<int4> fxt;
  for (int pass = 0; pass < 2; pass++)
    for (int k = 0; k < b->n; k++) {
      const af_ctx *h = b->inst[k];
      if ((h->opt.flux_limiter != 0) != (pass == 1)) continue;
      for (int j0 = 0; j0 < h->g.ny; j0 += FLUX_TY)
        for (int i0 = 0; i0 < h->g.nx; i0 += FLUX_TX) fxt.push_back(make_int4(k, i0, j0, 0));
    }
  int n_plain = 0;
  for (const int4 &t : fxt) n_plain += b->inst[t.x]->opt.flux_limiter ? 0 : 1;
  if (!b->d_fx_tiles) BCK(cudaMalloc(&b->d_fx_tiles, sizeof(int4) * fxt.size()), "batch: cudaMalloc(tiles)");
  BCK(cudaMemcpy(b->d_fx_tiles, fxt.data(), sizeof(int4) * fxt.size(), cudaMemcpyHostToDevice), "batch: tiles");
  b->n_fx_tiles = (int)fxt.size();
  // shock-indicator tiles of the instances with the blend on
  std::vector<int4> tht;
  for (int k = 0; k < b->n; k++) {
    const af_ctx *h = b->inst[k];
    if (!h->opt.shock_blend) continue;
    for (int b0 = 0; b0 <= h->g.ny + 1; b0 += 8)
      for (int a0 = 0; a0 <= h->g.nx + 1; a0 += 32) tht.push_back(make_int4(k, a0, b0, 0));
  }
  if ((int)tht.size() > b->theta_tiles_cap) {
    cudaFree(b->d_theta_tiles);
    b->d_theta_tiles = nullptr;
    BCK(cudaMalloc(&b->d_theta_tiles, sizeof(int4) * tht.size()), "batch: cudaMalloc(tiles)");
    b->theta_tiles_cap = (int)tht.size();
  }
  if (!tht.empty())
    BCK(cudaMemcpy(b->d_theta_tiles, tht.data(), sizeof(int4) * tht.size(), cudaMemcpyHostToDevice), "batch: tiles");
  const int n_theta = (int)tht.size();
  // captured launches differ
  if (any_lim != b->any_limiter || any_blend != b->any_blend || n_plain != b->n_fx_plain ||
      n_theta != b->n_theta_tiles)
    drop_graphs(b);
  b->n_theta_tiles = n_theta;
  b->n_fx_plain = n_plain;
  b->any_limiter = any_lim;
  b->any_blend = any_blend;
  return AF_OK;
}

// TMA descriptors and the point-value tile list for tile height b->tile_h
int build_tiles(af_batch *b) {
  if (b->maps_ok && b->pv_tiles_h == b->tile_h) return AF_OK;
  drop_graphs(b);
  std::vector<TileMaps> maps(2 * b->n);
  std::vector<int4> pv;
  for (int k = 0; k < b->n; k++) {
    af_ctx *h = b->inst[k];
    const Grid &g = h->g;
    for (int q = 0; q < 2; q++) {
      cudaError_t e = make_tile_maps(g, h->tbuf[q].k[VTX], h->tbuf[q].k[XE], h->tbuf[q].k[YE], h->hi, b->tile_h,
                                     &maps[2 * k + q]);
      if (e != cudaSuccess) return bcuda(e, "batch: TMA descriptors");
    }
    for (int j0 = 0; j0 < g.nyv; j0 += b->tile_h)
      for (int i0 = 0; i0 < g.nxv; i0 += 32) pv.push_back(make_int4(k, i0, j0, 0));
  }
  if (b->d_pv_tiles) cudaFree(b->d_pv_tiles);
  b->d_pv_tiles = nullptr;
  BCK(cudaMalloc(&b->d_pv_tiles, sizeof(int4) * pv.size()), "batch: cudaMalloc(tiles)");
  BCK(cudaMemcpy(b->d_pv_tiles, pv.data(), sizeof(int4) * pv.size(), cudaMemcpyHostToDevice), "batch: tiles");
  BCK(cudaMemcpy(b->d_maps, maps.data(), sizeof(TileMaps) * maps.size(), cudaMemcpyHostToDevice), "batch: maps");
  b->n_pv_tiles = (int)pv.size();
  b->pv_tiles_h = b->tile_h;
  b->maps_ok = true;
  return AF_OK;
}

PointValueBatch pv_batch(const af_batch *b) {
  PointValueBatch B;
  B.tiles = b->d_pv_tiles;
  B.ctl = b->d_ctl;
  B.args = b->d_pv;
  B.maps = b->d_maps;
  return B;
}

// what a step does before its point values: the ghost layers of t^n and the
// Sec. 3.4 blend weights (both functions of the t^n state alone)
int enqueue_pre_pointvalue(af_batch *b, cudaStream_t s) {
  GhostBatch G;
  G.ctl = b->d_ctl;
  G.grids = b->d_grids;
  G.arrays = b->d_arrays;
  G.chunks = b->d_ghost_chunks;
  BCK(launch_ghost_batch(G, b->n_ghost_chunks, s), "batch: ghost fill");
  if (b->any_blend)
    BCK(launch_shock_theta_batch(b->d_theta_tiles, b->n_theta_tiles, b->d_ctl, b->d_grids, b->d_arrays, b->d_theta,
                                 s),
        "batch: shock indicator");
  return AF_OK;
}

// one step of every active instance on stream s
int enqueue_batch_step(af_batch *b, double *hist, int hist_steps, cudaStream_t s) {
  BCK(launch_batch_dt(b->d_ctl, b->n, hist, hist_steps, DT_STEP, b->d_pv, s), "batch: dt");
  const int pre = enqueue_pre_pointvalue(b, s);
  if (pre) return pre;
  BCK(launch_pointvalue_batch(pv_batch(b), b->n_pv_tiles, b->tile_h, s), "batch: point values");
  if (b->sampling)
    BCK(launch_sample_batch(b->sampler, b->d_pv_tiles, b->n_pv_tiles, b->tile_h, b->d_ctl, b->d_pv, s),
        "batch: sampler");
  FluxBatch F;
  F.tiles = b->d_fx_tiles;
  F.ctl = b->d_ctl;
  F.args = b->d_fx;
  if (b->any_limiter) BCK(launch_snapshot_batch(F, b->n, s), "batch: flux limiter snapshot");
  BCK(launch_flux_batch(F, b->n_fx_plain, b->n_fx_tiles, s), "batch: flux update");
  return AF_OK;
}

// the graph of `steps` steps (and the closing buffer flip), captured once
int graph_for(af_batch *b, int steps, double *hist, int hist_steps, cudaGraphExec_t *out) {
  for (auto &e : b->graphs)
    if (e.steps == steps && e.hist == hist && e.hist_steps == hist_steps) {
      *out = e.exec;
      return AF_OK;
    }
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->own_stream, cudaStreamCaptureModeThreadLocal), "batch: capture");
  int rc = AF_OK;
  for (int k = 0; k < steps && rc == AF_OK; k++) rc = enqueue_batch_step(b, hist, hist_steps, b->own_stream);
  if (rc == AF_OK) {
    cudaError_t e = launch_batch_dt(b->d_ctl, b->n, hist, hist_steps, DT_SETTLE, b->d_pv, b->own_stream);
    if (e != cudaSuccess) rc = bcuda(e, "batch: settle");
  }
  cudaError_t e = cudaStreamEndCapture(b->own_stream, &graph);
  if (rc != AF_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return bcuda(e, "batch: capture");
  GraphEntry ent;
  e = cudaGraphInstantiate(&ent.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bcuda(e, "batch: instantiate");
  ent.steps = steps;
  ent.hist = hist;
  ent.hist_steps = hist_steps;
  if (b->graphs.size() >= 4) drop_graphs(b);
  b->graphs.push_back(ent);
  *out = ent.exec;
  return AF_OK;
}

// wave speeds of instances whose state was just set (the flux kernel keeps
// them current afterwards)
int ensure_speeds(af_batch *b) {
  for (int k = 0; k < b->n; k++) {
    if (b->speed_ok[k]) continue;
    af_ctx *h = b->inst[k];
    BatchCtl *c = b->d_ctl + k;
    BCK(launch_max_speed(h->g, h->hi, h->tbuf[b->ctl_h[k].cur], &c->speed, &c->speed_bad, b->stream),
        "batch: max speed");
    b->speed_ok[k] = 1;
  }
  return AF_OK;
}

void free_batch(af_batch *b) {
  drop_graphs(b);
  for (af_ctx *h : b->inst)
    if (h) af_destroy(h);
  cudaFree(b->d_ctl);
  cudaFree(b->d_pv);
  cudaFree(b->d_fx);
  cudaFree(b->d_maps);
  cudaFree(b->d_grids);
  cudaFree(b->d_ghost_chunks);
  cudaFree(b->d_theta_tiles);
  cudaFree(b->d_arrays);
  cudaFree(b->d_theta);
  cudaFree(b->d_pv_tiles);
  cudaFree(b->d_fx_tiles);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

}  // namespace

extern "C" {

af_batch *af_batch_create(int n, const int *nx, const int *ny, const double *dx, const double *dy,
                          double gamma, const uint32_t *bc) {
  if (n < 1 || n > 65535 || !nx || !ny || !dx || !dy || !bc) {
    bfail(AF_ERR_ARG, "af_batch_create: need 1 <= n <= 65535 and the size arrays");
    return nullptr;
  }
  af_batch *b = new (std::nothrow) af_batch();
  if (!b) {
    bfail(AF_ERR_ALLOC, "af_batch_create: out of host memory");
    return nullptr;
  }
  b->n = n;
  cudaGetDevice(&b->device);
  if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    bfail(AF_ERR_CUDA, "af_batch_create: stream");
    free_batch(b);
    return nullptr;
  }
  b->stream = b->own_stream;
  b->inst.assign(n, nullptr);
  for (int k = 0; k < n; k++) {
    b->inst[k] = af_create(nx[k], ny[k], dx[k], dy[k], gamma, bc[k]);
    if (!b->inst[k]) {  // af_create left its message
      free_batch(b);
      return nullptr;
    }
    af_set_stream(b->inst[k], b->stream);
  }
  b->ctl_h.assign(n, BatchCtl());
  b->has_state.assign(n, 0);
  b->speed_ok.assign(n, 0);
  b->stopped.assign(n, 0);
  std::vector<Grid> grids(n);
  std::vector<int4> chunks;
  for (int k = 0; k < n; k++) {
    BatchCtl &c = b->ctl_h[k];
    std::memset(&c, 0, sizeof(c));
    c.t_end = std::numeric_limits<double>::infinity();
    c.cfl = 0.3;
    c.dx = dx[k];
    c.dy = dy[k];
    c.h = dx[k] < dy[k] ? dx[k] : dy[k];
    c.cur = b->inst[k]->tmap_cur;
    grids[k] = b->inst[k]->g;
    for (int arr = 0; arr < 5; arr++)
      for (long long e = 0; e < ghost_total(grids[k], arr); e += GHOST_CHUNK)
        chunks.push_back(make_int4(k, arr, (int)e, 0));
  }
  b->n_ghost_chunks = (int)chunks.size();
  cudaError_t e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_pv, sizeof(PointValueArgs) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_fx, sizeof(FluxArgs) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_maps, sizeof(TileMaps) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_grids, sizeof(Grid) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_arrays, sizeof(float *) * 10 * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_theta, sizeof(float *) * 2 * n);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_grids, grids.data(), sizeof(Grid) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ghost_chunks, sizeof(int4) * chunks.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_ghost_chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    bcuda(e, "af_batch_create");
    free_batch(b);
    return nullptr;
  }
  if (put_ctl(b) != AF_OK || upload_args(b) != AF_OK || build_tiles(b) != AF_OK) {
    free_batch(b);
    return nullptr;
  }
  return b;
}

void af_batch_destroy(af_batch *b) {
  if (!b) return;
  Dev d(b->device);
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

int af_batch_set_stream(af_batch *b, void *stream) {
  if (!b) return bfail(AF_ERR_ARG, "null batch");
  Dev d(b->device);
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  b->stream = (cudaStream_t)stream;
  for (af_ctx *h : b->inst) af_set_stream(h, stream);
  return AF_OK;
}

int af_batch_set_option(af_batch *b, int k, int key, double value) {
  if (!b || k < -1 || k >= b->n) return bfail(AF_ERR_ARG, "af_batch_set_option: bad instance");
  if (key == AF_OPT_PROFILE) return bfail(AF_ERR_ARG, "af_batch_set_option: profiling is per handle");
  Dev d(b->device);
  const int k0 = k < 0 ? 0 : k, k1 = k < 0 ? b->n : k + 1;
  for (int q = k0; q < k1; q++) {
    int rc = af_set_option(b->inst[q], key, value);  // validates
    if (rc) return rc;
  }
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  if (key == AF_OPT_UBAR)  // the option lives in the grid description
    for (int q = k0; q < k1; q++)
      BCK(cudaMemcpy(b->d_grids + q, &b->inst[q]->g, sizeof(Grid), cudaMemcpyHostToDevice), "batch: grid");
  return upload_args(b);
}

int af_batch_set_inflow(af_batch *b, int k, int side, const double U[4]) {
  if (!b || k < 0 || k >= b->n) return bfail(AF_ERR_ARG, "af_batch_set_inflow: bad instance");
  Dev d(b->device);
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  int rc = af_set_inflow(b->inst[k], side, U);
  if (rc) return rc;
  BCK(cudaMemcpy(b->d_grids + k, &b->inst[k]->g, sizeof(Grid), cudaMemcpyHostToDevice), "batch: grid");
  return upload_args(b);  // the kernel arguments hold the grid description
}

int af_batch_set_state(af_batch *b, int k, const float *avg, const float *vtx, const float *xe,
                       const float *ye, void *stream) {
  if (!b || k < 0 || k >= b->n) return bfail(AF_ERR_ARG, "af_batch_set_state: bad instance");
  Dev d(b->device);
  int rc = sync_ctl(b);
  if (rc) return rc;
  rc = af_set_state(b->inst[k], avg, vtx, xe, ye, stream);
  if (rc) return rc;
  BatchCtl &c = b->ctl_h[k];
  c.t = 0.0;
  c.steps = 0;
  c.cur = b->inst[k]->tmap_cur;
  c.stepped = 0;
  c.status = 0;
  c.speed = 0;
  c.speed_bad = 0;
  std::memset(c.counters, 0, sizeof(c.counters));
  c.active = !(c.t_end <= 0.0);
  b->has_state[k] = 1;
  b->speed_ok[k] = 0;
  b->stopped[k] = 0;
  return put_ctl(b);
}

int af_batch_get_state(af_batch *b, int k, float *avg, float *vtx, float *xe, float *ye, void *stream) {
  if (!b || k < 0 || k >= b->n) return bfail(AF_ERR_ARG, "af_batch_get_state: bad instance");
  if (!b->has_state[k]) return bfail(AF_ERR_STATE, "af_batch_get_state: no state set");
  Dev d(b->device);
  int rc = sync_ctl(b);
  if (rc) return rc;
  return af_get_state(b->inst[k], avg, vtx, xe, ye, stream);
}

int af_batch_set_end(af_batch *b, const double *t_end, double cfl) {
  if (!b || !t_end) return bfail(AF_ERR_ARG, "af_batch_set_end: null argument");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return bfail(AF_ERR_ARG, "af_batch_set_end: cfl must be positive");
  for (int k = 0; k < b->n; k++)
    if (std::isnan(t_end[k])) return bfail(AF_ERR_ARG, "af_batch_set_end: end time is NaN");
  Dev d(b->device);
  int rc = sync_ctl(b);
  if (rc) return rc;
  for (int k = 0; k < b->n; k++) {
    BatchCtl &c = b->ctl_h[k];
    c.t_end = t_end[k];
    c.cfl = cfl;
    const bool before_end = std::isinf(c.t_end) ? c.t_end > 0 : (c.t_end - c.t) > 1e-12 * std::fabs(c.t_end);
    c.active = b->has_state[k] && !b->stopped[k] && before_end;
  }
  return put_ctl(b);
}

int af_batch_run(af_batch *b, int nsteps, double *hist, int hist_steps) {
  if (!b || nsteps < 0 || hist_steps < 0) return bfail(AF_ERR_ARG, "af_batch_run: bad arguments");
  for (int k = 0; k < b->n; k++)
    if (!b->has_state[k]) return bfail(AF_ERR_STATE, "af_batch_run: an instance has no state");
  if (b->timed_out)
    return bfail(AF_ERR_STATE, "af_batch_run: a wait for staged data timed out (AF_ST_TIMEOUT): the states are "
                               "invalid and the batch takes no further steps");
  if (nsteps == 0) return AF_OK;
  NvtxScope range("af_batch_run");
  Dev d(b->device);
  int rc = build_tiles(b);
  if (rc) return rc;
  rc = ensure_speeds(b);
  if (rc) return rc;
  int left = nsteps;
  while (left > 0) {
    const int steps = left > GRAPH_CHUNK ? GRAPH_CHUNK : left;
    cudaGraphExec_t ex = nullptr;
    rc = graph_for(b, steps, hist, hist_steps, &ex);
    if (rc) return rc;
    BCK(cudaGraphLaunch(ex, b->stream), "batch: graph launch");
    left -= steps;
  }
  return AF_OK;
}

int af_batch_query(af_batch *b, double *t, int *steps, int *active, int *status) {
  if (!b) return bfail(AF_ERR_ARG, "null batch");
  Dev d(b->device);
  int rc = sync_ctl(b);
  if (rc) return rc;
  for (int k = 0; k < b->n; k++) {
    const BatchCtl &c = b->ctl_h[k];
    if (t) t[k] = c.t;
    if (steps) steps[k] = c.steps;
    if (active) active[k] = c.active;
    if (status) status[k] = c.status;
  }
  if (status) {
    for (int k = 0; k < b->n; k++) b->ctl_h[k].status = 0;
    return put_ctl(b);
  }
  return AF_OK;
}

int af_batch_counters(af_batch *b, int64_t *out) {
  if (!b || !out) return bfail(AF_ERR_ARG, "null argument");
  Dev d(b->device);
  int rc = sync_ctl(b);
  if (rc) return rc;
  for (int k = 0; k < b->n; k++)
    for (int q = 0; q < 4; q++) out[4 * k + q] = (int64_t)b->ctl_h[k].counters[q];
  return AF_OK;
}

int af_batch_set_tile(af_batch *b, int tile_h) {
  if (!b) return bfail(AF_ERR_ARG, "null batch");
  if (tile_h != 4 && tile_h != 8 && tile_h != 16) return bfail(AF_ERR_ARG, "tile height must be 4, 8 or 16");
  Dev d(b->device);
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  b->tile_h = tile_h;
  return build_tiles(b);
}

int af_batch_autotune(af_batch *b, int *tile_h, double *ms) {
  if (!b) return bfail(AF_ERR_ARG, "null batch");
  for (int k = 0; k < b->n; k++)
    if (!b->has_state[k]) return bfail(AF_ERR_STATE, "af_batch_autotune: an instance has no state");
  Dev d(b->device);
  int rc = sync_ctl(b);
  if (rc) return rc;
  const std::vector<BatchCtl> saved = b->ctl_h;
  rc = ensure_speeds(b);
  if (rc) return rc;
  // the timed launches see what a step's point values see: ghost layers and
  // blend weights of the current state (both recomputed by every step)
  rc = enqueue_pre_pointvalue(b, b->stream);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "event");
  BCK(cudaEventCreate(&e1), "event");
  double best = 1e300;
  int best_h = b->tile_h;
  for (int c = 0; c < 3 && rc == AF_OK; c++) {
    b->tile_h = TILE_HEIGHTS[c];
    rc = build_tiles(b);
    if (rc) break;
    // dt of the coming step, nothing advanced
    cudaError_t e = launch_batch_dt(b->d_ctl, b->n, nullptr, 0, DT_PROBE, b->d_pv, b->stream);
    if (e == cudaSuccess) e = launch_pointvalue_batch(pv_batch(b), b->n_pv_tiles, b->tile_h, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    for (int r = 0; r < 3 && e == cudaSuccess; r++)
      e = launch_pointvalue_batch(pv_batch(b), b->n_pv_tiles, b->tile_h, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) {
      rc = bcuda(e, "af_batch_autotune");
      break;
    }
    if (ms) ms[c] = t / 3.0;
    if (t < best) {
      best = t;
      best_h = TILE_HEIGHTS[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timed launches touched only scratch levels, status and counters
  b->ctl_h = saved;
  if (rc) return rc;
  b->tile_h = best_h;
  rc = build_tiles(b);
  if (rc) return rc;
  for (int k = 0; k < b->n; k++) b->speed_ok[k] = 0;  // recomputed at the next run
  if (tile_h) *tile_h = best_h;
  return put_ctl(b);
}

int af_batch_set_sampler(af_batch *b, float *Xv, float *Tv, int *idv, int cap_v, float *Xe, float *Te, int *ide,
                         int cap_e, int *counts, uint64_t seed, double rate) {
  if (!b) return bfail(AF_ERR_ARG, "null batch");
  if (!(rate >= 0.0 && rate <= 1.0)) return bfail(AF_ERR_ARG, "af_batch_set_sampler: rate must be in [0, 1]");
  Dev d(b->device);
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  drop_graphs(b);
  if (rate == 0.0) {
    b->sampling = false;
    return AF_OK;
  }
  if (!Xv || !Tv || !Xe || !Te || !counts || cap_v < 0 || cap_e < 0)
    return bfail(AF_ERR_ARG, "af_batch_set_sampler: need the sample arrays and the counts");
  SampleBatch &S = b->sampler;
  S.X[0] = Xv;
  S.T[0] = Tv;
  S.id[0] = reinterpret_cast<int4 *>(idv);
  S.cap[0] = cap_v;
  S.X[1] = Xe;
  S.T[1] = Te;
  S.id[1] = reinterpret_cast<int4 *>(ide);
  S.cap[1] = cap_e;
  S.counts = counts;
  S.seed = seed;
  const double th = rate * 4294967296.0;
  S.threshold = th >= 4294967295.0 ? 0xFFFFFFFFu : (unsigned)th;
  b->sampling = true;
  return AF_OK;
}

long long af_batch_active_cells(af_batch *b) {
  if (!b) return bfail(AF_ERR_ARG, "null batch");
  Dev d(b->device);
  int rc = sync_ctl(b);
  if (rc) return rc;
  long long s = 0;
  for (int k = 0; k < b->n; k++)
    if (b->ctl_h[k].active) s += (long long)b->inst[k]->g.nx * b->inst[k]->g.ny;
  return s;
}

}  // extern "C"
