// af_api.cu -- the C ABI of include/af.h: handle, device state, transfers,
// step sequencing and reductions.  All numerical work is in the kernels of
// af_misc.cu, af_pointvalue.cu and af_flux.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/af.h"
#include "af_common.cuh"
#include "af_ctx.h"
#include "af_kernels.h"
#include "af_mlp.h"

using namespace af;

static thread_local char g_err[512] = "";

static int fail(int code, const char *fmt, const char *detail = nullptr) {
  std::snprintf(g_err, sizeof(g_err), fmt, detail ? detail : "");
  return code;
}
static int cuda_fail(cudaError_t e, const char *where) {
  std::snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
  return AF_ERR_CUDA;
}
int af::set_error(int code, const char *msg) {
  std::snprintf(g_err, sizeof(g_err), "%s", msg);
  return code;
}
#define CK(call, where)                         \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

namespace {

struct DeviceGuard {
  int old = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
    else old = -1;
  }
  ~DeviceGuard() {
    if (old >= 0) cudaSetDevice(old);
  }
};

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// make the handle's stream wait for `user`, or the reverse.  A null handle
// is a real stream here: the legacy default stream, which does not order
// itself with the handle's own (non-blocking) stream.
void order_after(af_ctx *h, cudaStream_t user) {
  if (user == h->stream) return;
  cudaEventRecord(h->ev_in, user);
  cudaStreamWaitEvent(h->stream, h->ev_in, 0);
}
void order_before(af_ctx *h, cudaStream_t user) {
  if (user == h->stream) return;
  cudaEventRecord(h->ev_out, h->stream);
  cudaStreamWaitEvent(user, h->ev_out, 0);
}

// external array extents of the four state arrays
void extents(const af_ctx *h, int which, int &ni, int &nj) {
  const int nx = h->g.nx, ny = h->g.ny;
  switch (which) {
    case 0: ni = nx; nj = ny; break;          // averages
    case 1: ni = nx + 1; nj = ny + 1; break;  // vertices
    case 2: ni = nx + 1; nj = ny; break;      // x-edges
    default: ni = nx; nj = ny + 1; break;     // y-edges
  }
}

int ensure_staging(af_ctx *h) {
  if (h->staging) return AF_OK;
  size_t off = 0;
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    h->staging_off[w] = off;
    off += ((size_t)NV * ni * nj + 63) / 64 * 64;  // 256-byte aligned areas
  }
  h->staging_off[4] = off;
  CK(cudaMalloc(&h->staging, off * sizeof(float)), "cudaMalloc(staging)");
  for (int w = 0; w < 4; w++) CK(cudaStreamCreateWithFlags(&h->xs[w], cudaStreamNonBlocking), "copy streams");
  for (int k = 0; k < 5; k++) CK(cudaEventCreateWithFlags(&h->xev[k], cudaEventDisableTiming), "copy events");
  return AF_OK;
}

// device external arrays -> padded planes (after the periodic-duplicate check)
int load_state(af_ctx *h, const float *const src[4]) {
  h->speed_valid = false;
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(h->d_bad, 0, sizeof(int), s), "memset");
  for (int w = 1; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    const int dup_x = h->g.per_x && (w == 1 || w == 2), dup_y = h->g.per_y && (w == 1 || w == 3);
    if (dup_x || dup_y) CK(launch_check_dup(src[w], ni, nj, dup_x, dup_y, h->d_bad, s), "check_dup");
  }
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, h->d_bad, sizeof(int), cudaMemcpyDeviceToHost, s), "memcpy");
  CK(cudaStreamSynchronize(s), "sync");
  if (bad) return fail(AF_ERR_ARG, "periodic state: the duplicated last node line differs from the first%s");
  float *dst[4] = {h->hi, h->lev[0].k[VTX], h->lev[0].k[XE], h->lev[0].k[YE]};
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    CK(launch_pack(h->g, src[w], dst[w], ni, nj, true, s), "pack");
  }
  CK(cudaMemsetAsync(h->lo, 0, sizeof(float) * NV * h->g.plane, s), "memset lo");
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), s), "memset status");
  h->has_state = true;
  h->half_valid = false;
  return AF_OK;
}

}  // namespace

extern "C" {

const char *af_last_error(void) { return g_err; }

af_ctx *af_create(int nx, int ny, double dx, double dy, double gamma, uint32_t bc) {
  if (nx < 2 || ny < 2 || !(dx > 0) || !(dy > 0) || !(gamma > 1.0) || !std::isfinite(dx) ||
      !std::isfinite(dy)) {
    fail(AF_ERR_ARG, "af_create: need nx, ny >= 2, dx, dy > 0 and gamma > 1%s");
    return nullptr;
  }
  int b[4];
  for (int k = 0; k < 4; k++) {
    b[k] = (int)((bc >> (8 * k)) & 0xffu);
    if (b[k] > AF_BC_INFLOW) {
      fail(AF_ERR_ARG, "af_create: unknown boundary kind%s");
      return nullptr;
    }
  }
  if ((b[0] == AF_BC_PERIODIC) != (b[1] == AF_BC_PERIODIC) ||
      (b[2] == AF_BC_PERIODIC) != (b[3] == AF_BC_PERIODIC)) {
    fail(AF_ERR_ARG, "af_create: periodic must be set on both sides of an axis%s");
    return nullptr;
  }
  if ((long long)nx * ny > (1LL << 31)) {
    fail(AF_ERR_ARG, "af_create: grid too large%s");
    return nullptr;
  }
  af_ctx *h = new (std::nothrow) af_ctx();
  if (!h) {
    fail(AF_ERR_ALLOC, "af_create: out of host memory%s");
    return nullptr;
  }
  Grid &g = h->g;
  g.nx = nx;
  g.ny = ny;
  g.P = ((nx + OX + G + 1) + 31) / 32 * 32;
  g.H = ny + OY + G + 1;
  g.plane = (long long)g.P * g.H;
  g.per_x = b[0] == AF_BC_PERIODIC;
  g.per_y = b[2] == AF_BC_PERIODIC;
  g.nxv = g.per_x ? nx : nx + 1;
  g.nyv = g.per_y ? ny : ny + 1;
  for (int k = 0; k < 4; k++) g.bc[k] = b[k];
  g.dx = (float)dx;
  g.dy = (float)dy;
  g.idx = (float)(1.0 / dx);
  g.idy = (float)(1.0 / dy);
  g.gamma = (float)gamma;
  for (int k = 0; k < 4; k++) {  // until set: rho = p = 1 at rest
    g.inflow[k][0] = g.inflow[k][3] = 1.0f;
    g.inflow[k][1] = g.inflow[k][2] = 0.0f;
  }
  h->dx = dx;
  h->dy = dy;
  h->gamma = gamma;
  cudaGetDevice(&h->device);
  // hi, lo, 3 levels x 3 node kinds and 4 node-flux arrays: 15 arrays of 4 planes
  const size_t state_bytes = 15 * (size_t)NV * (size_t)g.plane * sizeof(float);
  cudaError_t e = cudaMalloc(&h->base, state_bytes);
  if (e != cudaSuccess) {
    cuda_fail(e, "af_create: cudaMalloc(state)");
    delete h;
    return nullptr;
  }
  float *p = h->base;
  auto take = [&]() {
    float *q = p;
    p += (size_t)NV * g.plane;
    return q;
  };
  h->hi = take();
  h->lo = take();
  for (int l = 0; l < 3; l++)
    for (int k = 0; k < 3; k++) h->lev[l].k[k] = take();
  for (int q = 0; q < 4; q++) h->nflux[q] = take();
  h->tbuf[0] = h->lev[0];
  h->tbuf[1] = h->lev[2];
  h->tmap_cur = 0;
  {
    cudaError_t pe = prepare_pointvalue();
    if (pe != cudaSuccess) {
      cuda_fail(pe, "af_create: kernel attributes");
      cudaFree(h->base);
      delete h;
      return nullptr;
    }
  }
  for (int b = 0; b < 2; b++) {
    cudaError_t te = make_tile_maps(g, h->tbuf[b].k[VTX], h->tbuf[b].k[XE], h->tbuf[b].k[YE], h->hi, 8,
                                   &h->tmaps[b]);
    h->tile_h = 8;
    if (te != cudaSuccess) {
      cuda_fail(te, "af_create: TMA descriptors");
      cudaFree(h->base);
      delete h;
      return nullptr;
    }
  }
  const size_t small = 64 + 64 + 64 + 64 + sizeof(double) * (TOTALS_BLOCKS * NV + NV);
  e = cudaHostAlloc(&h->host_words, 64, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&h->host_words_dev, h->host_words, 0);
  if (e == cudaSuccess) e = cudaMalloc(&h->small, small);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
  for (int k = 0; k < 5 && e == cudaSuccess; k++) e = cudaEventCreate(&h->ev_stage[k]);
  if (e != cudaSuccess) {
    cuda_fail(e, "af_create");
    if (h->small) cudaFree(h->small);
    if (h->host_words) cudaFreeHost(h->host_words);
    cudaFree(h->base);
    delete h;
    return nullptr;
  }
  char *sp = (char *)h->small;
  h->d_status = (int *)sp;
  h->d_bad = (int *)(sp + 64);
  h->d_bad_async = (int *)(sp + 96);
  h->d_speed = (unsigned *)(sp + 128);
  h->d_speed_bad = (int *)(sp + 160);
  h->d_counters = (unsigned long long *)(sp + 192);
  h->d_min_keys = (unsigned *)(sp + 224);
  h->d_totals = (double *)(sp + 256);
  h->d_partials = h->d_totals + NV;
  h->stream = h->own_stream;
  // the whole state starts zeroed, ghosts included; checking builds fill it
  // with NaN instead, so that a read of a point no step or set call wrote
  // (a ghost layer not filled, padding) shows as a non-finite result
#ifdef AF_CHECK_BOUNDS
  cudaMemsetAsync(h->base, 0xFF, state_bytes, h->stream);
#else
  cudaMemsetAsync(h->base, 0, state_bytes, h->stream);
#endif
  cudaMemsetAsync(h->small, 0, small, h->stream);
  cudaStreamSynchronize(h->stream);
  return h;
}

void af_destroy(af_ctx *h) {
  if (!h) return;
  DeviceGuard dg(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->async_init) {
    for (int w = 0; w < 4; w++) cudaStreamSynchronize(h->xo[w]);
    cudaFree(h->staging_out);
    for (int w = 0; w < 4; w++) {
      cudaStreamDestroy(h->xo[w]);
      cudaEventDestroy(h->out_done[0][w]);
      cudaEventDestroy(h->out_done[1][w]);
    }
    cudaEventDestroy(h->in_free);
    cudaEventDestroy(h->out_ready);
  }
  if (h->staging) {
    for (int w = 0; w < 4; w++) cudaStreamSynchronize(h->xs[w]);
    cudaFree(h->staging);
    for (int w = 0; w < 4; w++) cudaStreamDestroy(h->xs[w]);
    for (int k = 0; k < 5; k++) cudaEventDestroy(h->xev[k]);
  }
  for (int p = 0; p < 2; p++)
    if (h->run_exec[p]) cudaGraphExecDestroy(h->run_exec[p]);
  cudaFree(h->small);
  if (h->host_words) cudaFreeHost(h->host_words);
  cudaFree(h->base);
  if (h->surr_ubar) cudaFree(h->surr_ubar);
  if (h->shock_theta) cudaFree(h->shock_theta);
  if (h->q0) cudaFree(h->q0);
  if (h->f64_base) cudaFree(h->f64_base);
  cudaEventDestroy(h->ev_in);
  cudaEventDestroy(h->ev_out);
  for (int k = 0; k < 5; k++) cudaEventDestroy(h->ev_stage[k]);
  cudaStreamDestroy(h->own_stream);
  delete h;
}

int af_set_stream(af_ctx *h, void *stream) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  cudaStream_t s = (cudaStream_t)stream;
  if (s != h->stream) {
    DeviceGuard dg(h->device);
    order_after(h, s);  // new stream starts after everything queued so far
    cudaStream_t old = h->stream;
    h->stream = s;
    order_after(h, old);
  }
  return AF_OK;
}

int af_set_option(af_ctx *h, int key, double value) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  const int iv = (int)value;
  switch (key) {
    case AF_OPT_LIN_MODE:
      if (iv < 0 || iv > 2) return fail(AF_ERR_ARG, "lin_mode must be 0, 1 or 2%s");
      h->opt.lin_mode = iv;
      return AF_OK;
    case AF_OPT_TSW: h->opt.tsw = iv != 0; return AF_OK;
    case AF_OPT_LIMITER: h->opt.limiter = iv != 0; return AF_OK;
    case AF_OPT_CORRECTION: h->opt.correction = iv != 0; return AF_OK;
    case AF_OPT_FORCE_LO:
      if (iv < 0 || iv > 2) return fail(AF_ERR_ARG, "force_lo must be 0, 1 or 2%s");
      h->opt.force_lo = iv;
      return AF_OK;
    case AF_OPT_PROFILE: h->profile = iv != 0; return AF_OK;
    case AF_OPT_SURROGATE:
      if (iv && (!h->surr[0] || !h->surr[1])) return fail(AF_ERR_STATE, "no surrogate networks set%s");
      h->opt.surrogate = iv != 0;
      return AF_OK;
    case AF_OPT_SURR_TOL:
      if (!(value >= 0.0) || !std::isfinite(value)) return fail(AF_ERR_ARG, "surrogate tolerance must be >= 0%s");
      h->opt.surr_tol = (float)value;
      return AF_OK;
    case AF_OPT_FLUX_LIMITER:
      if (iv && !h->q0) {
        DeviceGuard dg(h->device);
        CK(cudaMalloc(&h->q0, sizeof(float) * NV * (size_t)h->g.plane), "cudaMalloc(flux limiter snapshot)");
      }
      h->opt.flux_limiter = iv != 0;
      return AF_OK;
    case AF_OPT_SHOCK_BLEND:
      if (iv && !h->shock_theta) {
        DeviceGuard dg(h->device);
        CK(cudaMalloc(&h->shock_theta, 2 * sizeof(float) * (size_t)h->g.plane), "cudaMalloc(theta)");
        CK(cudaMemset(h->shock_theta, 0, 2 * sizeof(float) * (size_t)h->g.plane), "memset(theta)");
      }
      h->opt.shock_blend = iv != 0;
      return AF_OK;
    case AF_OPT_NODE_BOUNDS: h->opt.node_bounds = iv != 0; return AF_OK;
    case AF_OPT_TEST_TIMEOUT: h->opt.test_timeout = iv != 0; return AF_OK;
    case AF_OPT_NODE_FLUX: h->opt.node_flux = iv != 0; return AF_OK;
    case AF_OPT_FP64: {
      const bool on = iv != 0;
      if (on && !h->f64_base) {
        DeviceGuard dg(h->device);
        // averages (4 planes), 3 levels x 3 node arrays (36 planes), records
        // (40 doubles a cell), then the reduction words
        const size_t planes = (40 + REC64_DOUBLES) * (size_t)h->g.plane;
        const size_t bytes = sizeof(double) * (planes + TOTALS64_PARTIALS + 4) + 64;
        CK(cudaMalloc(&h->f64_base, bytes), "cudaMalloc(FP64 state)");
        double *p = h->f64_base;
        h->f64_avg = p;
        p += NV * (size_t)h->g.plane;
        for (int l = 0; l < 3; l++)
          for (int k = 0; k < 3; k++) {
            h->f64_lev[l][k] = p;
            p += NV * (size_t)h->g.plane;
          }
        h->f64_rec = p;
        p += REC64_DOUBLES * (size_t)h->g.plane;
        h->f64_partials = p;
        p += TOTALS64_PARTIALS;
        h->f64_totals = p;
        p += 4;
        h->f64_speed = reinterpret_cast<unsigned long long *>(p);
        h->f64_bad = reinterpret_cast<int *>(p + 1);
      }
      if (on != h->fp64) h->has_state = false;  // a state of the other precision is not carried over
      h->fp64 = on;
      return AF_OK;
    }
    case AF_OPT_KEEP_HALF:
      if ((iv != 0) != (h->keep_half != 0)) {
        for (int p = 0; p < 2; p++)  // captured steps hold the old launch arguments
          if (h->run_exec[p]) {
            DeviceGuard dg(h->device);
            cudaGraphExecDestroy(h->run_exec[p]);
            h->run_exec[p] = nullptr;
          }
      }
      h->keep_half = iv != 0;
      return AF_OK;
    case AF_OPT_UBAR:
      if (iv < 0 || iv > 1) return fail(AF_ERR_ARG, "ubar must be 0 or 1%s");
      if (iv != h->g.ubar_c2p) {
        for (int p = 0; p < 2; p++)  // captured steps hold the old grid description
          if (h->run_exec[p]) {
            DeviceGuard dg(h->device);
            cudaGraphExecDestroy(h->run_exec[p]);
            h->run_exec[p] = nullptr;
          }
      }
      h->g.ubar_c2p = iv;
      return AF_OK;
    case AF_OPT_TILE_H: {
      if (iv != 4 && iv != 8 && iv != 16) return fail(AF_ERR_ARG, "tile height must be 4, 8 or 16%s");
      if (iv == h->tile_h) return AF_OK;
      DeviceGuard dg(h->device);
      CK(cudaStreamSynchronize(h->stream), "sync");
      for (int b = 0; b < 2; b++)
        CK(make_tile_maps(h->g, h->tbuf[b].k[VTX], h->tbuf[b].k[XE], h->tbuf[b].k[YE], h->hi, iv, &h->tmaps[b]),
           "TMA descriptors");
      h->tile_h = iv;
      for (int p = 0; p < 2; p++)  // captured steps hold the old launch shape
        if (h->run_exec[p]) {
          cudaGraphExecDestroy(h->run_exec[p]);
          h->run_exec[p] = nullptr;
        }
      return AF_OK;
    }
    case AF_OPT_SURR_ABS:
      if (!(value >= 0.0) || !std::isfinite(value)) return fail(AF_ERR_ARG, "surrogate tolerance must be >= 0%s");
      h->opt.surr_abs = (float)value;
      return AF_OK;
    case AF_OPT_SURR_SMOOTH:
      if (!(value >= 0.0)) return fail(AF_ERR_ARG, "surrogate stencil limit must be >= 0%s");
      h->opt.surr_smooth = value > 3.0e38 ? 3.0e38f : (float)value;
      return AF_OK;
    default: return fail(AF_ERR_ARG, "unknown option%s");
  }
}

int af_get_option(af_ctx *h, int key, double *value) {
  if (!h || !value) return fail(AF_ERR_ARG, "null argument%s");
  switch (key) {
    case AF_OPT_LIN_MODE: *value = h->opt.lin_mode; return AF_OK;
    case AF_OPT_TSW: *value = h->opt.tsw; return AF_OK;
    case AF_OPT_LIMITER: *value = h->opt.limiter; return AF_OK;
    case AF_OPT_CORRECTION: *value = h->opt.correction; return AF_OK;
    case AF_OPT_FORCE_LO: *value = h->opt.force_lo; return AF_OK;
    case AF_OPT_PROFILE: *value = h->profile; return AF_OK;
    case AF_OPT_SURROGATE: *value = h->opt.surrogate; return AF_OK;
    case AF_OPT_SURR_TOL: *value = h->opt.surr_tol; return AF_OK;
    case AF_OPT_SURR_ABS: *value = h->opt.surr_abs; return AF_OK;
    case AF_OPT_SURR_SMOOTH: *value = h->opt.surr_smooth; return AF_OK;
    case AF_OPT_FLUX_LIMITER: *value = h->opt.flux_limiter; return AF_OK;
    case AF_OPT_SHOCK_BLEND: *value = h->opt.shock_blend; return AF_OK;
    case AF_OPT_NODE_BOUNDS: *value = h->opt.node_bounds; return AF_OK;
    case AF_OPT_UBAR: *value = h->g.ubar_c2p; return AF_OK;
    case AF_OPT_TEST_TIMEOUT: *value = h->opt.test_timeout; return AF_OK;
    case AF_OPT_KEEP_HALF: *value = h->keep_half; return AF_OK;
    case AF_OPT_NODE_FLUX: *value = h->opt.node_flux; return AF_OK;
    case AF_OPT_FP64: *value = h->fp64 ? 1.0 : 0.0; return AF_OK;
    case AF_OPT_TILE_H: *value = h->tile_h; return AF_OK;
    default: return fail(AF_ERR_ARG, "unknown option%s");
  }
}

int af_set_state(af_ctx *h, const float *avg, const float *vtx, const float *xe, const float *ye,
                 void *stream) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (h->fp64) return fail(AF_ERR_STATE, "the handle is in FP64 mode: use af_set_state_f64%s");
  DeviceGuard dg(h->device);
  const float *src[4] = {avg, vtx, xe, ye};
  for (int w = 0; w < 4; w++)
    if (!is_device_ptr(src[w])) return fail(AF_ERR_ARG, "af_set_state: arrays must be device memory%s");
  order_after(h, (cudaStream_t)stream);
  int rc = load_state(h, src);
  order_before(h, (cudaStream_t)stream);
  return rc;
}

int af_set_state_host(af_ctx *h, const float *avg, const float *vtx, const float *xe,
                      const float *ye) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (h->async_pending) {
    const int rc = af_host_sync(h);
    if (rc) return rc;
  }
  h->speed_valid = false;
  if (!avg || !vtx || !xe || !ye) return fail(AF_ERR_ARG, "af_set_state_host: null array%s");
  DeviceGuard dg(h->device);
  int rc = ensure_staging(h);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  const float *src[4] = {avg, vtx, xe, ye};
  float *dst[4] = {h->hi, h->lev[0].k[VTX], h->lev[0].k[XE], h->lev[0].k[YE]};
  CK(cudaMemsetAsync(h->d_bad, 0, sizeof(int), s), "memset");
  // the four copies run on their own streams once the handle's stream has
  // reached this point; each array is checked and packed when it has arrived
  CK(cudaEventRecord(h->xev[4], s), "event");
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    CK(cudaStreamWaitEvent(h->xs[w], h->xev[4], 0), "event");
    CK(cudaMemcpyAsync(h->staging + h->staging_off[w], src[w], sizeof(float) * NV * ni * nj,
                       cudaMemcpyHostToDevice, h->xs[w]),
       "af_set_state_host: H2D");
    CK(cudaEventRecord(h->xev[w], h->xs[w]), "event");
  }
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    float *stg = h->staging + h->staging_off[w];
    CK(cudaStreamWaitEvent(s, h->xev[w], 0), "event");
    const int dup_x = h->g.per_x && (w == 1 || w == 2), dup_y = h->g.per_y && (w == 1 || w == 3);
    if (dup_x || dup_y) CK(launch_check_dup(stg, ni, nj, dup_x, dup_y, h->d_bad, s), "check_dup");
    CK(launch_pack(h->g, stg, dst[w], ni, nj, true, s), "pack");
  }
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, h->d_bad, sizeof(int), cudaMemcpyDeviceToHost, s), "memcpy");
  CK(cudaMemsetAsync(h->lo, 0, sizeof(float) * NV * h->g.plane, s), "memset lo");
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), s), "memset status");
  CK(cudaStreamSynchronize(s), "sync");
  if (bad) {
    h->has_state = false;
    return fail(AF_ERR_ARG, "periodic state: the duplicated last node line differs from the first%s");
  }
  h->has_state = true;
  h->half_valid = false;
  return AF_OK;
}

static int get_arrays(af_ctx *h, NodeSet &ns, const float *avgsrc, float *dst[4], bool host,
                      cudaStream_t user) {
  const float *src[4] = {avgsrc, ns.k[VTX], ns.k[XE], ns.k[YE]};
  cudaStream_t s = h->stream;
  if (!host) {
    for (int w = 0; w < 4; w++)
      if (dst[w] && !is_device_ptr(dst[w])) return fail(AF_ERR_ARG, "arrays must be device memory%s");
    order_after(h, user);
  } else {
    int rc = ensure_staging(h);
    if (rc) return rc;
  }
  for (int w = 0; w < 4; w++) {
    if (!dst[w] || !src[w]) continue;
    int ni, nj;
    extents(h, w, ni, nj);
    if (!host) {
      CK(launch_pack(h->g, src[w], dst[w], ni, nj, false, s), "pack");
    } else {
      // pack on the handle's stream, copy out on the array's own stream
      float *stg = h->staging + h->staging_off[w];
      CK(launch_pack(h->g, src[w], stg, ni, nj, false, s), "pack");
      CK(cudaEventRecord(h->xev[w], s), "event");
      CK(cudaStreamWaitEvent(h->xs[w], h->xev[w], 0), "event");
      CK(cudaMemcpyAsync(dst[w], stg, sizeof(float) * NV * ni * nj, cudaMemcpyDeviceToHost, h->xs[w]), "D2H");
    }
  }
  if (host)
    for (int w = 0; w < 4; w++) CK(cudaStreamSynchronize(h->xs[w]), "sync");
  if (!host) order_before(h, user);
  return AF_OK;
}

int af_get_state(af_ctx *h, float *avg, float *vtx, float *xe, float *ye, void *stream) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (h->fp64) return fail(AF_ERR_STATE, "the handle is in FP64 mode: use af_get_state_f64%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  DeviceGuard dg(h->device);
  float *dst[4] = {avg, vtx, xe, ye};
  return get_arrays(h, h->lev[0], h->hi, dst, false, (cudaStream_t)stream);
}

// FP64 path: the compact arrays of af_set_state / af_get_state in double
// (device memory), packed into or out of the padded FP64 planes
int af_set_state_f64(af_ctx *h, const double *avg, const double *vtx, const double *xe, const double *ye,
                     void *stream) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!h->fp64) return fail(AF_ERR_STATE, "af_set_state_f64: turn AF_OPT_FP64 on first%s");
  const double *src[4] = {avg, vtx, xe, ye};
  for (int w = 0; w < 4; w++)
    if (!is_device_ptr(src[w])) return fail(AF_ERR_ARG, "af_set_state_f64: arrays must be device memory%s");
  DeviceGuard dg(h->device);
  order_after(h, (cudaStream_t)stream);
  double *dst[4] = {h->f64_avg, h->f64_lev[0][VTX], h->f64_lev[0][XE], h->f64_lev[0][YE]};
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    CK(launch_pack64(h->g, src[w], dst[w], ni, nj, true, h->stream), "pack");
  }
  order_before(h, (cudaStream_t)stream);
  h->has_state = true;
  h->half_valid = false;
  return AF_OK;
}

int af_get_state_f64(af_ctx *h, double *avg, double *vtx, double *xe, double *ye, void *stream) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!h->fp64) return fail(AF_ERR_STATE, "af_get_state_f64: the handle is not in FP64 mode%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  double *dst[4] = {avg, vtx, xe, ye};
  for (int w = 0; w < 4; w++)
    if (!is_device_ptr(dst[w])) return fail(AF_ERR_ARG, "af_get_state_f64: arrays must be device memory%s");
  DeviceGuard dg(h->device);
  order_after(h, (cudaStream_t)stream);
  const double *src[4] = {h->f64_avg, h->f64_lev[0][VTX], h->f64_lev[0][XE], h->f64_lev[0][YE]};
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    CK(launch_pack64(h->g, src[w], dst[w], ni, nj, false, h->stream), "unpack");
  }
  order_before(h, (cudaStream_t)stream);
  return AF_OK;
}

int af_get_state_host(af_ctx *h, float *avg, float *vtx, float *xe, float *ye) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  if (h->async_pending) {
    const int rc = af_host_sync(h);
    if (rc) return rc;
  }
  DeviceGuard dg(h->device);
  float *dst[4] = {avg, vtx, xe, ye};
  return get_arrays(h, h->lev[0], h->hi, dst, true, nullptr);
}

// ---------------------------------------------------------------- asynchronous host transfers
static int ensure_async(af_ctx *h) {
  int rc = ensure_staging(h);
  if (rc) return rc;
  if (h->async_init) return AF_OK;
  CK(cudaMalloc(&h->staging_out, 2 * h->staging_off[4] * sizeof(float)), "cudaMalloc(download staging)");
  for (int w = 0; w < 4; w++) {
    CK(cudaStreamCreateWithFlags(&h->xo[w], cudaStreamNonBlocking), "copy streams");
    for (int b = 0; b < 2; b++)
      CK(cudaEventCreateWithFlags(&h->out_done[b][w], cudaEventDisableTiming), "copy events");
  }
  CK(cudaEventCreateWithFlags(&h->in_free, cudaEventDisableTiming), "copy events");
  CK(cudaEventCreateWithFlags(&h->out_ready, cudaEventDisableTiming), "copy events");
  // nothing is pending yet: the first waits on these pass at once
  CK(cudaEventRecord(h->in_free, h->stream), "event");
  for (int w = 0; w < 4; w++)
    for (int b = 0; b < 2; b++) CK(cudaEventRecord(h->out_done[b][w], h->xo[w]), "event");
  h->out_slot = 0;
  h->async_init = true;
  return AF_OK;
}

int af_set_state_host_async(af_ctx *h, const float *avg, const float *vtx, const float *xe,
                            const float *ye) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!avg || !vtx || !xe || !ye) return fail(AF_ERR_ARG, "af_set_state_host_async: null array%s");
  DeviceGuard dg(h->device);
  int rc = ensure_async(h);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  const float *src[4] = {avg, vtx, xe, ye};
  float *dst[4] = {h->hi, h->lev[0].k[VTX], h->lev[0].k[XE], h->lev[0].k[YE]};
  // each copy waits until the previous upload's unpack has read the staging
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    CK(cudaStreamWaitEvent(h->xs[w], h->in_free, 0), "event");
    CK(cudaMemcpyAsync(h->staging + h->staging_off[w], src[w], sizeof(float) * NV * ni * nj,
                       cudaMemcpyHostToDevice, h->xs[w]),
       "af_set_state_host_async: H2D");
    CK(cudaEventRecord(h->xev[w], h->xs[w]), "event");
  }
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    float *stg = h->staging + h->staging_off[w];
    CK(cudaStreamWaitEvent(s, h->xev[w], 0), "event");
    const int dup_x = h->g.per_x && (w == 1 || w == 2), dup_y = h->g.per_y && (w == 1 || w == 3);
    if (dup_x || dup_y) CK(launch_check_dup(stg, ni, nj, dup_x, dup_y, h->d_bad_async, s), "check_dup");
    CK(launch_pack(h->g, stg, dst[w], ni, nj, true, s), "pack");
  }
  CK(cudaEventRecord(h->in_free, s), "event");
  CK(cudaMemsetAsync(h->lo, 0, sizeof(float) * NV * h->g.plane, s), "memset lo");
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), s), "memset status");
  h->speed_valid = false;
  h->has_state = true;
  h->half_valid = false;
  h->async_pending = true;
  return AF_OK;
}

int af_get_state_host_async(af_ctx *h, float *avg, float *vtx, float *xe, float *ye) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  if (!avg || !vtx || !xe || !ye) return fail(AF_ERR_ARG, "af_get_state_host_async: null array%s");
  DeviceGuard dg(h->device);
  int rc = ensure_async(h);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  float *dst[4] = {avg, vtx, xe, ye};
  const float *src[4] = {h->hi, h->lev[0].k[VTX], h->lev[0].k[XE], h->lev[0].k[YE]};
  // pack into the download staging area used two downloads ago, once that
  // download has left it
  const int b = h->out_slot;
  float *stg = h->staging_out + (size_t)b * h->staging_off[4];
  for (int w = 0; w < 4; w++) CK(cudaStreamWaitEvent(s, h->out_done[b][w], 0), "event");
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    CK(launch_pack(h->g, src[w], stg + h->staging_off[w], ni, nj, false, s), "pack");
  }
  CK(cudaEventRecord(h->out_ready, s), "event");
  for (int w = 0; w < 4; w++) {
    int ni, nj;
    extents(h, w, ni, nj);
    CK(cudaStreamWaitEvent(h->xo[w], h->out_ready, 0), "event");
    CK(cudaMemcpyAsync(dst[w], stg + h->staging_off[w], sizeof(float) * NV * ni * nj, cudaMemcpyDeviceToHost,
                       h->xo[w]),
       "af_get_state_host_async: D2H");
    CK(cudaEventRecord(h->out_done[b][w], h->xo[w]), "event");
  }
  h->out_slot = b ^ 1;
  h->async_pending = true;
  return AF_OK;
}

int af_host_sync(af_ctx *h) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!h->async_init) return AF_OK;
  DeviceGuard dg(h->device);
  for (int w = 0; w < 4; w++) CK(cudaStreamSynchronize(h->xs[w]), "sync");
  for (int w = 0; w < 4; w++) CK(cudaStreamSynchronize(h->xo[w]), "sync");
  CK(cudaStreamSynchronize(h->stream), "sync");
  h->async_pending = false;
  int bad = 0;
  CK(cudaMemcpy(&bad, h->d_bad_async, sizeof(int), cudaMemcpyDeviceToHost), "memcpy");
  if (bad) {
    CK(cudaMemset(h->d_bad_async, 0, sizeof(int)), "memset");
    h->has_state = false;
    return fail(AF_ERR_ARG, "periodic state: the duplicated last node line differs from the first%s");
  }
  return AF_OK;
}

int af_get_half(af_ctx *h, float *vtx, float *xe, float *ye, void *stream) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  if (!h->half_valid)
    return fail(AF_ERR_STATE, "af_get_half: the last step kept no t^{n+1/2} level (set AF_OPT_KEEP_HALF before it)%s");
  DeviceGuard dg(h->device);
  float *dst[4] = {nullptr, vtx, xe, ye};
  return get_arrays(h, h->lev[1], nullptr, dst, false, (cudaStream_t)stream);
}

int af_get_avg_lo(af_ctx *h, float *avg_lo, void *stream) {
  if (!h || !is_device_ptr(avg_lo)) return fail(AF_ERR_ARG, "af_get_avg_lo: need a device array%s");
  DeviceGuard dg(h->device);
  order_after(h, (cudaStream_t)stream);
  CK(launch_pack(h->g, h->lo, avg_lo, h->g.nx, h->g.ny, false, h->stream), "pack");
  order_before(h, (cudaStream_t)stream);
  return AF_OK;
}

int af_set_avg_lo(af_ctx *h, const float *avg_lo, void *stream) {
  h->speed_valid = false;
  if (!h || !is_device_ptr(avg_lo)) return fail(AF_ERR_ARG, "af_set_avg_lo: need a device array%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  DeviceGuard dg(h->device);
  order_after(h, (cudaStream_t)stream);
  CK(launch_pack(h->g, avg_lo, h->lo, h->g.nx, h->g.ny, true, h->stream), "pack");
  order_before(h, (cudaStream_t)stream);
  return AF_OK;
}

// fold the stage times of the previous profiled step into the totals
static void collect_stages(af_ctx *h) {
  if (!h->stage_pending) return;
  cudaEventSynchronize(h->ev_stage[4]);
  // events: 0 | prep | 1 | point values | 2 | (none) | 3 | flux | 4
  const int from[3] = {0, 1, 3}, to[3] = {1, 2, 4};
  for (int k = 0; k < 3; k++) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->ev_stage[from[k]], h->ev_stage[to[k]]) == cudaSuccess) h->stage_ms[k] += ms;
  }
  h->stage_pending = false;
}

static int enqueue_step(af_ctx *h, double dt) {
  cudaStream_t s = h->stream;
  const bool prof = h->profile != 0;
  if (prof) {
    collect_stages(h);
    cudaEventRecord(h->ev_stage[0], s);
  }
  {
    NvtxScope st("ghost fill");
    CK(launch_ghost_fill(h->g, h->hi, h->lo, h->lev[0], s), "ghost fill");
  }
  h->launches[AF_STAGE_PREP] += 1;
  CK(cudaMemsetAsync(h->d_counters, 0, 4 * sizeof(unsigned long long), s), "memset counters");
  const float *theta[2] = {nullptr, nullptr};
  if (h->opt.shock_blend) {
    theta[0] = h->shock_theta;
    theta[1] = h->shock_theta + h->g.plane;
    CK(launch_shock_theta(h->g, h->hi, h->lev[0], h->shock_theta, h->shock_theta + h->g.plane, s),
       "shock indicator");
  }
  if (prof) cudaEventRecord(h->ev_stage[1], s);
  {
    NvtxScope pvr("point values");
    if (h->opt.surrogate) {
      // network at every node, then the exact operator at the nodes it rejected
      CK(cudaMemsetAsync(h->surr_tiles, 0, sizeof(int) * h->surr_tiles_x * ((h->g.nyv + h->tile_h - 1) / h->tile_h), s),
         "memset tiles");
      CK(launch_ubar(h->g, h->hi, h->lev[0], h->surr_ubar, s), "surrogate cell prep");
      const unsigned char *mask[3];
      for (int k = 0; k < 3; k++) {
        SurrogateArgs A;
        A.g = h->g;
        for (int q = 0; q < 3; q++) {
          A.n0[q] = h->lev[0].k[q];
          A.n1[q] = h->lev[1].k[q];
          A.n2[q] = h->lev[2].k[q];
        }
        A.hi = h->hi;
        A.ubar = h->surr_ubar;
        A.dt = (float)dt;
        A.tol = h->opt.surr_tol;
        A.tol_abs = h->opt.surr_abs;
        A.smooth = h->opt.surr_smooth;
        af_mlp *net = h->surr[k == VTX ? 0 : 1];
        A.wb = net->wb;
        A.params = net->params;
        A.mask = h->surr_mask + (size_t)k * h->g.plane;
        mask[k] = A.mask;
        A.tile_flag = h->surr_tiles;
        A.tiles_x = h->surr_tiles_x;
        A.tile_rows = h->tile_h;
        A.stats = h->surr_stats;
        A.status = h->d_status;
        A.test_no_issue = h->opt.test_timeout != 0;
        A.wait_limit = h->opt.test_timeout ? kTestWaitLimit : kWaitLimit;
        CK(launch_surrogate(k, A, h->sms, s), "surrogate");
      }
      CK(launch_pointvalue_masked(h->g, h->lev[0], h->hi, h->tmaps[h->tmap_cur], h->lev[1], h->lev[2], (float)dt,
                                  h->opt, h->d_status, h->d_counters, mask, h->surr_tiles, theta, h->tile_h, s),
         "point values (fallback)");
      h->launches[AF_STAGE_POINTVALUE] += 5;
      h->half_valid = true;
    } else if (!h->opt.node_flux) {
      // plain path: t^{n+1/2} and t^{n+1} written, the flux kernel forms the
      // node fluxes from three levels
      CK(launch_pointvalue(h->g, h->lev[0], h->hi, h->tmaps[h->tmap_cur], h->lev[1], h->lev[2], (float)dt,
                           h->opt, h->d_status, h->d_counters, theta, h->tile_h, nullptr, s),
         "point values");
      h->launches[AF_STAGE_POINTVALUE] += 1;
      h->half_valid = true;
    } else {
      // node-flux path: the point-value kernel writes the node fluxes (and
      // folds the new point values into the wave speed) for the flux kernel
      NodeFluxOut nf;
      for (int q = 0; q < 4; q++) nf.q[q] = h->nflux[q];
      nf.speed = h->d_speed;
      nf.speed_bad = h->d_speed_bad;
      nf.write_half = h->keep_half;
      CK(cudaMemsetAsync(h->d_speed, 0, sizeof(unsigned), s), "memset speed");
      CK(cudaMemsetAsync(h->d_speed_bad, 0, sizeof(int), s), "memset speed");
      CK(launch_pointvalue(h->g, h->lev[0], h->hi, h->tmaps[h->tmap_cur], h->lev[1], h->lev[2], (float)dt,
                           h->opt, h->d_status, h->d_counters, theta, h->tile_h, &nf, s),
         "point values");
      h->launches[AF_STAGE_POINTVALUE] += 1;
      h->half_valid = h->keep_half != 0;
    }
  }
  if (prof) {
    cudaEventRecord(h->ev_stage[2], s);
    cudaEventRecord(h->ev_stage[3], s);
  }
  NvtxScope fl("flux update");
  // the limiter reads t^n averages while the kernel overwrites them: snapshot
  if (h->opt.flux_limiter)
    CK(cudaMemcpyAsync(h->q0, h->hi, sizeof(float) * NV * (size_t)h->g.plane, cudaMemcpyDeviceToDevice, s),
       "flux limiter snapshot");
  if (h->opt.surrogate || !h->opt.node_flux) {
    CK(launch_flux_update(h->g, h->lev[0], h->lev[1], h->lev[2], h->hi, h->lo, dt / h->dx, dt / h->dy,
                          h->d_status, h->d_speed, h->d_speed_bad, h->opt.flux_limiter, h->q0, s),
       "flux update");
  } else {
    const float *nf[4] = {h->nflux[0], h->nflux[1], h->nflux[2], h->nflux[3]};
    CK(launch_flux_nf(h->g, nf, h->hi, h->lo, dt / h->dx, dt / h->dy, h->d_status, h->d_speed, h->d_speed_bad,
                      h->opt.flux_limiter, h->q0, s),
       "flux update");
  }
  h->speed_valid = true;
  h->launches[AF_STAGE_FLUX] += 1;
  if (prof) {
    cudaEventRecord(h->ev_stage[4], s);
    h->stage_pending = true;
  }
  NodeSet t = h->lev[0];
  h->lev[0] = h->lev[2];
  h->lev[2] = t;
  h->tmap_cur ^= 1;
  return AF_OK;
}

static const char *kTimedOut =
    "a wait for staged data or for the tensor cores timed out (AF_ST_TIMEOUT): the state is invalid and the "
    "handle takes no further steps%s";

// one step of the FP64 path: ghost layers, cell records, point values, fluxes
static int step64(af_ctx *h, double dt) {
  const Options &o = h->opt;
  if (o.tsw || o.limiter || o.force_lo || o.surrogate || o.flux_limiter || o.shock_blend || o.node_bounds ||
      o.node_flux)
    return fail(AF_ERR_STATE,
                "the FP64 path has no Sec. 3 limiters or switches: set tsw, limiter, force_lo, surrogate, "
                "flux_limiter, shock_blend, node_bounds and node_flux to 0%s");
  for (int k = 0; k < 4; k++)
    if (h->g.bc[k] == AF_BC_INFLOW) return fail(AF_ERR_STATE, "the FP64 path has no inflow sides%s");
  cudaStream_t s = h->stream;
  CK(launch_ghost_fill64(h->g, h->f64_avg, h->f64_lev[0], s), "FP64 ghost fill");
  Step64 S;
  S.g = h->g;
  S.ph.gam = h->gamma;
  S.ph.dx = h->dx;
  S.ph.dy = h->dy;
  S.avg = h->f64_avg;
  for (int k = 0; k < 3; k++) {
    S.n0[k] = h->f64_lev[0][k];
    S.n1[k] = h->f64_lev[1][k];
    S.n2[k] = h->f64_lev[2][k];
  }
  S.recs = h->f64_rec;
  S.dt = dt;
  S.lin_mode = o.lin_mode;
  S.correction = o.correction;
  S.status = h->d_status;
  CK(launch_step64(S, dt / h->dx, dt / h->dy, s), "FP64 step");
  for (int k = 0; k < 3; k++) std::swap(h->f64_lev[0][k], h->f64_lev[2][k]);
  return AF_OK;
}

int af_step(af_ctx *h, double dt) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(AF_ERR_ARG, "af_step: dt must be positive%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  if (h->timed_out) return fail(AF_ERR_STATE, kTimedOut);
  NvtxScope range("af_step");
  if (h->fp64) {
    DeviceGuard dg(h->device);
    return step64(h, dt);
  }
  DeviceGuard dg(h->device);
  return enqueue_step(h, dt);
}

static bool same_options(const Options &a, const Options &b) {
  return a.lin_mode == b.lin_mode && a.tsw == b.tsw && a.limiter == b.limiter &&
         a.correction == b.correction && a.force_lo == b.force_lo && a.surrogate == b.surrogate &&
         a.surr_tol == b.surr_tol && a.surr_abs == b.surr_abs && a.surr_smooth == b.surr_smooth &&
         a.flux_limiter == b.flux_limiter &&
         a.shock_blend == b.shock_blend && a.node_bounds == b.node_bounds && a.test_timeout == b.test_timeout &&
         a.node_flux == b.node_flux;
}

// Capture two steps on the handle's own stream (the t^n and t^{n+1} buffers
// swap every step, so after two steps every pointer is back where it was).
static int capture_pair(af_ctx *h, double dt) {
  const int p = h->tmap_cur;
  if (h->run_exec[p]) {
    cudaGraphExecDestroy(h->run_exec[p]);
    h->run_exec[p] = nullptr;
  }
  cudaStream_t keep = h->stream;
  const int keep_prof = h->profile;
  h->stream = h->own_stream;
  h->profile = 0;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->own_stream, cudaStreamCaptureModeThreadLocal);
  int rc = AF_OK;
  if (e == cudaSuccess) {
    rc = enqueue_step(h, dt);
    if (rc == AF_OK) rc = enqueue_step(h, dt);
    e = cudaStreamEndCapture(h->own_stream, &graph);
  }
  h->stream = keep;
  h->profile = keep_prof;
  if (rc != AF_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "af_run: capture");
  e = cudaGraphInstantiate(&h->run_exec[p], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "af_run: instantiate");
  h->run_dt[p] = dt;
  h->run_opt[p] = h->opt;
  return AF_OK;
}

int af_run(af_ctx *h, int nsteps, double dt) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(AF_ERR_ARG, "af_run: bad arguments%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  if (h->timed_out) return fail(AF_ERR_STATE, kTimedOut);
  NvtxScope range("af_run");
  DeviceGuard dg(h->device);
  if (h->fp64) {
    for (int k = 0; k < nsteps; k++) {
      int rc = step64(h, dt);
      if (rc) return rc;
    }
    return AF_OK;
  }
  if (h->profile || nsteps < 4) {  // profiled runs time every stage: plain launches
    for (int k = 0; k < nsteps; k++) {
      int rc = enqueue_step(h, dt);
      if (rc) return rc;
    }
    return AF_OK;
  }
  const int p = h->tmap_cur;
  if (!h->run_exec[p] || h->run_dt[p] != dt || !same_options(h->run_opt[p], h->opt)) {
    NvtxScope cap("af_run/capture");
    int rc = capture_pair(h, dt);
    if (rc) return rc;
  }
  for (int k = 0; k + 1 < nsteps; k += 2) {
    CK(cudaGraphLaunch(h->run_exec[p], h->stream), "af_run: graph launch");
    h->launches[AF_STAGE_PREP] += 2;
    h->launches[AF_STAGE_POINTVALUE] += h->opt.surrogate ? 10 : 2;
    h->launches[AF_STAGE_FLUX] += 2;
  }
  h->speed_valid = true;
  if (nsteps & 1) return enqueue_step(h, dt);
  return AF_OK;
}

int af_debug_bounds(unsigned *out) {
  if (!out) return fail(AF_ERR_ARG, "null argument%s");
  CK(cudaDeviceSynchronize(), "af_debug_bounds: sync");
  *out = af::bounds_flux() | af::bounds_fp64() | af::bounds_misc() | af::bounds_pointvalue() | af::bounds_surrogate();
#ifdef AF_CHECK_BOUNDS
  return 1;
#else
  return 0;
#endif
}

int af_status(af_ctx *h) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  DeviceGuard dg(h->device);
  CK(launch_export_words(reinterpret_cast<unsigned *>(h->d_status), nullptr, 1, h->host_words_dev, h->stream),
     "status");
  CK(cudaStreamSynchronize(h->stream), "sync");
  const int bits = (int)reinterpret_cast<volatile unsigned *>(h->host_words)[0];
  if (bits & AF_ST_TIMEOUT) h->timed_out = true;
  return h->timed_out ? bits | AF_ST_TIMEOUT : bits;  // sticky
}

int af_counters(af_ctx *h, int64_t out[4]) {
  if (!h || !out) return fail(AF_ERR_ARG, "null argument%s");
  DeviceGuard dg(h->device);
  unsigned long long c[4];
  CK(cudaMemcpyAsync(c, h->d_counters, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "counters");
  CK(cudaStreamSynchronize(h->stream), "sync");
  for (int k = 0; k < 4; k++) out[k] = (int64_t)c[k];
  return AF_OK;
}

int af_conserved_totals(af_ctx *h, double out[4]) {
  if (!h || !out) return fail(AF_ERR_ARG, "null argument%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  DeviceGuard dg(h->device);
  if (h->fp64) {
    CK(launch_totals64(h->g, h->f64_avg, h->f64_partials, h->dx * h->dy, h->f64_totals, h->stream), "totals");
    CK(cudaMemcpyAsync(out, h->f64_totals, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "totals");
    CK(cudaStreamSynchronize(h->stream), "sync");
    return AF_OK;
  }
  CK(launch_totals(h->g, h->hi, h->lo, h->d_partials, h->d_totals, h->stream), "totals");
  h->launches[AF_STAGE_REDUCE] += 2;
  double t[4];
  CK(cudaMemcpyAsync(t, h->d_totals, sizeof(t), cudaMemcpyDeviceToHost, h->stream), "totals");
  CK(cudaStreamSynchronize(h->stream), "sync");
  for (int v = 0; v < 4; v++) out[v] = t[v] * h->dx * h->dy;
  return AF_OK;
}

// the max-speed words, through mapped host memory (no copy engine: a large
// asynchronous download must not delay this read)
static cudaError_t read_speed(af_ctx *h, unsigned &bits, int &bad) {
  cudaError_t e = launch_export_words(h->d_speed, reinterpret_cast<unsigned *>(h->d_speed_bad), 0,
                                      h->host_words_dev, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  volatile unsigned *w = h->host_words;
  bits = w[0];
  bad = (int)w[1];
  return cudaSuccess;
}

int af_state_min(af_ctx *h, float out[2]) {
  if (!h || !out) return fail(AF_ERR_ARG, "null argument%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  if (h->fp64) return fail(AF_ERR_STATE, "af_state_min: the FP64 state has no FP32 minima (use af_get_state_f64)%s");
  DeviceGuard dg(h->device);
  CK(launch_state_min(h->g, h->hi, h->lev[0], h->d_min_keys, h->stream), "state minima");
  unsigned keys[3];
  CK(cudaMemcpyAsync(keys, h->d_min_keys, sizeof(keys), cudaMemcpyDeviceToHost, h->stream), "state minima");
  CK(cudaStreamSynchronize(h->stream), "sync");
  for (int q = 0; q < 2; q++) {
    const unsigned u = (keys[q] & 0x80000000u) ? (keys[q] & 0x7FFFFFFFu) : ~keys[q];
    std::memcpy(&out[q], &u, sizeof(float));
    if (keys[2]) out[q] = NAN;
  }
  return AF_OK;
}

int af_max_speed(af_ctx *h, float *out) {
  if (!h || !out) return fail(AF_ERR_ARG, "null argument%s");
  if (!h->has_state) return fail(AF_ERR_STATE, "no state set%s");
  DeviceGuard dg(h->device);
  if (h->fp64) {
    const double *n[3] = {h->f64_lev[0][VTX], h->f64_lev[0][XE], h->f64_lev[0][YE]};
    CK(launch_speed64(h->g, h->gamma, h->f64_avg, n, h->f64_speed, h->f64_bad, h->stream), "FP64 max speed");
    unsigned long long bits = 0;
    int bad = 0;
    CK(cudaMemcpyAsync(&bits, h->f64_speed, sizeof(bits), cudaMemcpyDeviceToHost, h->stream), "speed");
    CK(cudaMemcpyAsync(&bad, h->f64_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream), "speed");
    CK(cudaStreamSynchronize(h->stream), "sync");
    double m;
    std::memcpy(&m, &bits, sizeof(m));
    *out = bad ? NAN : (float)m;
    return AF_OK;
  }
  if (h->speed_valid) {  // computed by the last step's flux kernel
    unsigned bits = 0;
    int bad = 0;
    CK(read_speed(h, bits, bad), "speed");
    float m;
    std::memcpy(&m, &bits, sizeof(m));
    *out = bad ? NAN : m;
    return AF_OK;
  }
  cudaEvent_t e0 = h->ev_in, e1 = h->ev_out;
  if (h->profile) {
    collect_stages(h);
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    cudaEventRecord(e0, h->stream);
  }
  CK(launch_max_speed(h->g, h->hi, h->lev[0], h->d_speed, h->d_speed_bad, h->stream), "max speed");
  h->launches[AF_STAGE_REDUCE] += 1;
  if (h->profile) cudaEventRecord(e1, h->stream);
  unsigned bits = 0;
  int bad = 0;
  CK(read_speed(h, bits, bad), "speed");
  if (h->profile) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) h->stage_ms[AF_STAGE_REDUCE] += ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  float m;
  std::memcpy(&m, &bits, sizeof(m));
  *out = bad ? NAN : m;
  h->speed_valid = true;
  return AF_OK;
}

int af_profile(af_ctx *h, double ms[4], int64_t launches[4], int reset) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream), "sync");
  collect_stages(h);
  for (int k = 0; k < 4; k++) {
    if (ms) ms[k] = h->stage_ms[k];
    if (launches) launches[k] = h->launches[k];
    if (reset) {
      h->stage_ms[k] = 0.0;
      h->launches[k] = 0;
    }
  }
  return AF_OK;
}

int af_set_inflow(af_ctx *h, int side, const double U[4]) {
  if (!h || side < 0 || side > 3 || !U) return fail(AF_ERR_ARG, "af_set_inflow: bad arguments%s");
  if (!(U[0] > 0.0) || !(U[3] > 0.0) || !std::isfinite(U[1]) || !std::isfinite(U[2]))
    return fail(AF_ERR_ARG, "af_set_inflow: the state must have rho, p > 0%s");
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream), "sync");
  for (int v = 0; v < NV; v++) h->g.inflow[side][v] = (float)U[v];
  for (int p = 0; p < 2; p++)  // captured steps hold the old grid description
    if (h->run_exec[p]) {
      cudaGraphExecDestroy(h->run_exec[p]);
      h->run_exec[p] = nullptr;
    }
  return AF_OK;
}

int af_set_surrogate(af_ctx *h, af_mlp *vertex_net, af_mlp *edge_net) {
  if (!h) return fail(AF_ERR_ARG, "null handle%s");
  if (!vertex_net != !edge_net) return fail(AF_ERR_ARG, "af_set_surrogate: give both networks or neither%s");
  if (vertex_net && std::fabs(h->dx - h->dy) > 1e-12 * h->dx)
    return fail(AF_ERR_ARG, "af_set_surrogate: the surrogate needs square cells (dx = dy)%s");
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (vertex_net && !h->surr_mask) {
    const int tx = (h->g.nxv + 31) / 32, ty = (h->g.nyv + 3) / 4;  // enough for every tile height
    const size_t mask_bytes = (3 * (size_t)h->g.plane + 255) & ~size_t(255);
    const size_t ub_bytes = sizeof(float) * NV * (size_t)h->g.plane;
    // the 64-bit counters after the tile flags start on a 256-byte boundary
    // (tx * ty is odd on some grids: 65 x 513 tiles for 2049 x 2049 nodes)
    const size_t tile_bytes = (sizeof(int) * (size_t)tx * ty + 255) & ~size_t(255);
    const size_t bytes = ub_bytes + mask_bytes + tile_bytes + 2 * sizeof(unsigned long long);
    void *p = nullptr;
    CK(cudaMalloc(&p, bytes), "af_set_surrogate: cudaMalloc");
    cudaMemset(p, 0, bytes);
    h->surr_ubar = (float *)p;
    h->surr_mask = (unsigned char *)p + ub_bytes;
    h->surr_tiles = (int *)((char *)h->surr_mask + mask_bytes);
    h->surr_ntiles = tx * ty;
    h->surr_tiles_x = tx;
    h->surr_stats = (unsigned long long *)((char *)h->surr_tiles + tile_bytes);
    CK(prepare_surrogate(), "af_set_surrogate: kernel attributes");
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  }
  h->surr[0] = vertex_net;
  h->surr[1] = edge_net;
  if (!vertex_net) h->opt.surrogate = 0;
  for (int p = 0; p < 2; p++)  // captured steps hold the old networks
    if (h->run_exec[p]) {
      cudaGraphExecDestroy(h->run_exec[p]);
      h->run_exec[p] = nullptr;
    }
  return AF_OK;
}

int af_surrogate_stats(af_ctx *h, int64_t out[2], int reset) {
  if (!h || !out) return fail(AF_ERR_ARG, "null argument%s");
  if (!h->surr_stats) {
    out[0] = out[1] = 0;
    return AF_OK;
  }
  DeviceGuard dg(h->device);
  unsigned long long c[2];
  CK(cudaMemcpyAsync(c, h->surr_stats, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "stats");
  if (reset) CK(cudaMemsetAsync(h->surr_stats, 0, sizeof(c), h->stream), "stats");
  CK(cudaStreamSynchronize(h->stream), "sync");
  out[0] = (int64_t)c[0];
  out[1] = (int64_t)c[1];
  return AF_OK;
}

}  // extern "C"
