// C ABI entry points: context, workspace, launch accounting, validation and
// the whole-pair driver (Alg. 4).
#include <cstring>
#include <mutex>

#include "internal.h"

namespace cdl {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* msg, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", msg, file, line);
}

int ws_get(cdl_ctx* ctx, const char* name, size_t bytes, void** out) {
  if (bytes == 0) bytes = 256;
  auto it = ctx->ws.find(name);
  if (it != ctx->ws.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return CDL_OK;
  }
  size_t old = 0;
  if (it != ctx->ws.end()) {
    old = it->second.second;
    CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    CDL_CUDA_TRY(cudaFree(it->second.first));
    ctx->ws_used -= old;
    ctx->ws.erase(it);
  }
  if (ctx->ws_cap && ctx->ws_used + bytes > ctx->ws_cap) return CDL_ERR_OOM;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CDL_ERR_OOM;
  }
  ctx->ws_used += bytes;
  ctx->ws[name] = {p, bytes};
  *out = p;
  return CDL_OK;
}

static cudaEvent_t take_event(cdl_ctx* ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

Launch::Launch(cdl_ctx* c, int k, double w) : ctx(c), kc(k), work(w) {
  if (ctx->timing) {
    a = take_event(ctx);
    cudaEventRecord(a, ctx->stream);
  }
}

int Launch::done() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e), "kernel launch", kc);
    return CDL_ERR_CUDA;
  }
  ctx->launches += 1;
  ctx->kc_launches[kc] += 1;
  ctx->kc_work[kc] += work;
  if (ctx->timing) {
    cudaEvent_t b = take_event(ctx);
    cudaEventRecord(b, ctx->stream);
    Event2 ev;
    ev.a = a;
    ev.b = b;
    ev.kc = kc;
    ev.work = work;
    ctx->pending.push_back(ev);
  }
  return CDL_OK;
}

CopyTimer::CopyTimer(cdl_ctx* c, cudaStream_t st, double b) : ctx(c), s(st), bytes(b) {
  if (ctx->timing) {
    a = take_event(ctx);
    cudaEventRecord(a, s);
  }
}

void CopyTimer::done() {
  ctx->kc_launches[CDL_KC_HOST_LINK] += 1;
  ctx->kc_work[CDL_KC_HOST_LINK] += bytes;
  if (ctx->timing) {
    cudaEvent_t b = take_event(ctx);
    cudaEventRecord(b, s);
    Event2 ev;
    ev.a = a;
    ev.b = b;
    ev.kc = CDL_KC_HOST_LINK;
    ev.work = bytes;
    ctx->pending.push_back(ev);
  }
}

static int fold_timing(cdl_ctx* ctx) {
  if (ctx->pending.empty()) return CDL_OK;
  CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (auto& ev : ctx->pending) {
    float ms = 0.f;
    cudaEventSynchronize(ev.b);   // copies run on a chain's own copy stream
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    ctx->kc_ms[ev.kc] += ms;
    ctx->free_events.push_back(ev.a);
    ctx->free_events.push_back(ev.b);
  }
  ctx->pending.clear();
  return CDL_OK;
}

static int check_device_ptr(const void* p, int device) {
  if (!p) return CDL_ERR_INVALID_ARG;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return CDL_ERR_INVALID_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return CDL_ERR_INVALID_ARG;
  if (at.type == cudaMemoryTypeDevice && at.device != device) return CDL_ERR_INVALID_ARG;
  return CDL_OK;
}

static int check_aligned(const void* p, size_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) ? CDL_ERR_INVALID_ARG : CDL_OK;
}

static int dev_ptr(const cdl_ctx* ctx, const void* p, size_t align = 8) {
  CDL_TRY(check_device_ptr(p, ctx->device));
  return check_aligned(p, align);
}

int check_dev_ptr(const cdl_ctx* ctx, const void* p, size_t align) { return dev_ptr(ctx, p, align); }

int ctx_absorb(cdl_ctx* dst, cdl_ctx* src) {
  CDL_TRY(fold_timing(src));
  dst->launches += src->launches;
  src->launches = 0;
  for (int i = 0; i < CDL_KC_COUNT; ++i) {
    dst->kc_ms[i] += src->kc_ms[i];
    dst->kc_launches[i] += src->kc_launches[i];
    dst->kc_work[i] += src->kc_work[i];
    src->kc_ms[i] = 0;
    src->kc_launches[i] = 0;
    src->kc_work[i] = 0;
  }
  return CDL_OK;
}

static int set_device(cdl_ctx* ctx) {
  CDL_CUDA_TRY(cudaSetDevice(ctx->device));
  return CDL_OK;
}

int chain_create_regen(cdl_ctx* ctx, int64_t n, int d, int resident, cdl_chain** out) {
  if (!tc_supported(ctx)) return CDL_ERR_UNSUPPORTED;
  const int64_t npad = round_up(n, 256);
  cdl_chain* ch = new cdl_chain();
  ch->device = ctx->device;
  ch->n = n;
  ch->npad = npad;
  ch->d = d;
  ch->d_eff = d;
  ch->dtype = CDL_BF16;
  ch->elem = 2;
  ch->resident = resident;
  const double one = 1.0;
  if (ooc_init(ch) != CDL_OK || cudaMalloc(&ch->a_scale, 2 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ch->rsqrt_d, npad * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ch->D, npad * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ch->vol, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cdl_chain_free(ch);
    return CDL_ERR_OOM;
  }
  // Gaussian-kernel graphs: A <= 1, so the exact slices are taken of A itself
  // (a_scale[0] = 1) and 1 bounds max A (a_scale[1], the projection's grids)
  if (cudaMemcpy(ch->a_scale, &one, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ch->a_scale + 1, &one, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cdl_chain_free(ch);
    return CDL_ERR_CUDA;
  }
  *out = ch;
  return CDL_OK;
}
}  // namespace cdl

using namespace cdl;

extern "C" {

const char* cdl_status_string(int s) {
  switch (s) {
    case CDL_OK: return "CDL_OK";
    case CDL_ERR_INVALID_ARG: return "CDL_ERR_INVALID_ARG";
    case CDL_ERR_OOM: return "CDL_ERR_OOM";
    case CDL_ERR_CUDA: return "CDL_ERR_CUDA";
    case CDL_ERR_NOT_CONVERGED: return "CDL_ERR_NOT_CONVERGED";
    case CDL_ERR_TIMEOUT: return "CDL_ERR_TIMEOUT";
    case CDL_ERR_UNSUPPORTED: return "CDL_ERR_UNSUPPORTED";
    default: return "CDL_ERR_UNKNOWN";
  }
}

// Last CUDA error text recorded by this thread (diagnostics; not in cdl.h).
const char* cdl_last_error_detail(void) { return g_last_error; }

int cdl_ctx_create(cdl_ctx** out, int device, void* cuda_stream, size_t ws_cap_bytes) {
  if (!out) return CDL_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  const cudaError_t de = cudaGetDeviceCount(&ndev);
  if (de != cudaSuccess) {
    set_last_error(cudaGetErrorString(de), __FILE__, __LINE__);
    cudaGetLastError();
    return CDL_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return CDL_ERR_INVALID_ARG;
  CDL_CUDA_TRY(cudaSetDevice(device));
  cdl_ctx* ctx = new cdl_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->ws_cap = ws_cap_bytes;
  if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&ctx->dev_status, 256) != cudaSuccess ||
      cudaMemset(ctx->dev_status, 0, 256) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return CDL_ERR_CUDA;
  }
  *out = ctx;
  return CDL_OK;
}

int cdl_ctx_destroy(cdl_ctx* ctx) {
  if (!ctx) return CDL_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pair_chain) cdl_chain_free(ctx->pair_chain);
  if (ctx->regen_chain) cdl_chain_free(ctx->regen_chain);
  if (ctx->batch) batch_plan_free(ctx->batch);
  for (auto& kv : ctx->ws) cudaFree(kv.second.first);
  for (auto& ev : ctx->pending) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  cudaFree(ctx->dev_status);
  delete ctx;
  return CDL_OK;
}

int cdl_sync(cdl_ctx* ctx) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  CDL_TRY(set_device(ctx));
  CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  unsigned st = 0;
  CDL_CUDA_TRY(cudaMemcpy(&st, ctx->dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st != DEV_OK) {
    CDL_CUDA_TRY(cudaMemset(ctx->dev_status, 0, sizeof(unsigned)));
    return CDL_ERR_TIMEOUT;
  }
  return CDL_OK;
}

int cdl_ctx_set_timing(cdl_ctx* ctx, int enable) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  CDL_TRY(fold_timing(ctx));
  ctx->timing = enable != 0;
  return CDL_OK;
}

int cdl_ctx_timing(cdl_ctx* ctx, int kc, double* total_ms, int64_t* launches, double* work) {
  if (!ctx || kc < 0 || kc >= CDL_KC_COUNT) return CDL_ERR_INVALID_ARG;
  CDL_TRY(set_device(ctx));
  CDL_TRY(fold_timing(ctx));
  if (total_ms) *total_ms = ctx->kc_ms[kc];
  if (launches) *launches = ctx->kc_launches[kc];
  if (work) *work = ctx->kc_work[kc];
  return CDL_OK;
}

int cdl_ctx_reset_counters(cdl_ctx* ctx) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  CDL_TRY(set_device(ctx));
  CDL_TRY(fold_timing(ctx));
  ctx->launches = 0;
  for (int i = 0; i < CDL_KC_COUNT; ++i) {
    ctx->kc_ms[i] = 0;
    ctx->kc_launches[i] = 0;
    ctx->kc_work[i] = 0;
  }
  return CDL_OK;
}

int cdl_ctx_set_debug(cdl_ctx* ctx, int flags) {
  if (!ctx || (flags & ~(CDL_DEBUG_WITHHOLD_TC_LOAD | CDL_DEBUG_BATCH_VARIANT | 0xFF00))) return CDL_ERR_INVALID_ARG;
  ctx->debug_flags = flags;
  return CDL_OK;
}

int cdl_ctx_launch_count(cdl_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return CDL_ERR_INVALID_ARG;
  *launches = ctx->launches;
  return CDL_OK;
}

int cdl_build_graph(cdl_ctx* ctx, const double* X, int64_t n, int32_t T, double sigma,
                    cdl_dtype a_dtype, void* A, double* D, double* vol, double* sigma_out) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || T < 1 || T > 4096) return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, X));
  CDL_TRY(dev_ptr(ctx, A));
  CDL_TRY(dev_ptr(ctx, D));
  CDL_TRY(dev_ptr(ctx, vol));
  CDL_TRY(dev_ptr(ctx, sigma_out));
  return graph_build(ctx, X, n, T, sigma, static_cast<double*>(A), D, vol, sigma_out, CDL_KERNEL_GAUSSIAN);
}

int cdl_build_graph_kernel(cdl_ctx* ctx, const double* X, int64_t n, int32_t T, int32_t kernel, double sigma,
                           cdl_dtype a_dtype, void* A, double* D, double* vol, double* sigma_out) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  if (kernel != CDL_KERNEL_GAUSSIAN && kernel != CDL_KERNEL_EXP) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || T < 1 || T > 4096) return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, X));
  CDL_TRY(dev_ptr(ctx, A));
  CDL_TRY(dev_ptr(ctx, D));
  CDL_TRY(dev_ptr(ctx, vol));
  CDL_TRY(dev_ptr(ctx, sigma_out));
  return graph_build(ctx, X, n, T, sigma, static_cast<double*>(A), D, vol, sigma_out, kernel);
}

int cdl_graph_degrees(cdl_ctx* ctx, const void* A, cdl_dtype a_dtype, int64_t n, double* D, double* vol) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  if (n < 1 || n > (1 << 20)) return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A));
  CDL_TRY(dev_ptr(ctx, D));
  CDL_TRY(dev_ptr(ctx, vol));
  return graph_degrees(ctx, static_cast<const double*>(A), n, D, vol);
}

int cdl_graph_add_edges(cdl_ctx* ctx, void* A, cdl_dtype a_dtype, int64_t n, int64_t m, const int64_t* ij,
                        const double* w, int64_t* n_bad) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || m < 0) return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A));
  if (m > 0) {
    CDL_TRY(dev_ptr(ctx, ij));
    CDL_TRY(dev_ptr(ctx, w));
  }
  return graph_add_edges(ctx, static_cast<double*>(A), n, m, ij, w, n_bad);
}

int cdl_build_graph_static(const double* X, int64_t n, int32_t T, double sigma, double* A,
                           double* D, double* vol, double* sigma_out, void* cuda_stream) {
  return graph_build_static(X, n, T, sigma, A, D, vol, sigma_out, static_cast<cudaStream_t>(cuda_stream));
}

int cdl_chain_free(cdl_chain* ch) {
  if (!ch) return CDL_OK;
  cudaSetDevice(ch->device);
  if (ch->host_levels)
    ooc_destroy(ch);
  else
    cudaFree(ch->levels);
  cudaFree(ch->aop);
  cudaFree(ch->levels16);
  cudaFree(ch->amax);
  cudaFree(ch->ahl);
  cudaFree(ch->aslices);
  cudaFree(ch->a_scale);
  cudaFree(ch->tscale);
  cudaFree(ch->tatoms);
  cudaFree(ch->rsqrt_d);
  cudaFree(ch->D);
  cudaFree(ch->vol);
  delete ch;
  return CDL_OK;
}

int cdl_chain_depth(const cdl_chain* ch, int32_t* d_eff) {
  if (!ch || !d_eff) return CDL_ERR_INVALID_ARG;
  *d_eff = ch->d_eff;
  return CDL_OK;
}

int cdl_chain_level(const cdl_chain* ch, int32_t i, void** level, int64_t* npad) {
  if (!ch || i < 0 || i >= ch->d_eff) return CDL_ERR_INVALID_ARG;
  if (ch->host_levels && ch->copy) CDL_CUDA_TRY(cudaStreamSynchronize(ch->copy));   // copies to the host complete
  if (level) *level = ch->host_levels ? ooc_level_ptr(ch, i) : ch->level(i);
  if (npad) *npad = ch->npad;
  return CDL_OK;
}

int cdl_chain_apply_level(const cdl_chain* ch, int32_t i, void** level) {
  if (!level) return CDL_ERR_INVALID_ARG;
  *level = nullptr;
  if (!ch || i < 0 || i >= ch->d) return CDL_ERR_INVALID_ARG;
  if (ch->dtype != CDL_BF16 && ch->dtype != CDL_FP8E4M3 && ch->dtype != CDL_FP8E4M3_T128) return CDL_ERR_INVALID_ARG;
  *level = ch->level16(i);
  return CDL_OK;
}

int cdl_chain_tile_scales(const cdl_chain* ch, int32_t i, float** scales, int64_t* nt) {
  if (!ch || !scales || i < 0 || i >= ch->d || ch->dtype != CDL_FP8E4M3_T128) return CDL_ERR_INVALID_ARG;
  const int64_t t = ch->npad / 128;
  *scales = ch->tscale + (size_t)i * t * t;
  if (nt) *nt = t;
  return CDL_OK;
}

int cdl_chain_level_scale(const cdl_chain* ch, int32_t i, double* scale) {
  if (!ch || !scale || i < 0 || i >= ch->d) return CDL_ERR_INVALID_ARG;
  *scale = 1.0;
  if (ch->dtype != CDL_FP8E4M3) return CDL_OK;
  CDL_CUDA_TRY(cudaSetDevice(ch->device));
  CDL_CUDA_TRY(cudaDeviceSynchronize());
  unsigned bits = 0;
  CDL_CUDA_TRY(cudaMemcpy(&bits, ch->amax + i, sizeof(unsigned), cudaMemcpyDeviceToHost));
  float a;
  std::memcpy(&a, &bits, sizeof(float));
  *scale = a > 0.f ? (double)(a * (1.0f / 448.0f)) : 1.0;
  return CDL_OK;
}

int cdl_chain_build(cdl_ctx* ctx, const void* A, cdl_dtype a_dtype, const double* D,
                    const double* vol, int64_t n, int32_t d, cdl_dtype chain_dtype,
                    int32_t flags, cdl_chain** inout) {
  if (!ctx || !inout) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || d < 1 || d > 64 ||
      (flags & ~(CDL_CHAIN_HOST_LEVELS | CDL_CHAIN_TRUNCATE | CDL_CHAIN_RESIDENT_MASK)))
    return CDL_ERR_INVALID_ARG;
  const bool host_levels = (flags & CDL_CHAIN_HOST_LEVELS) != 0;
  const int resident = (flags & CDL_CHAIN_RESIDENT_MASK) >> CDL_CHAIN_RESIDENT_SHIFT;
  if (resident && !host_levels) return CDL_ERR_INVALID_ARG;
  const bool truncate = (flags & CDL_CHAIN_TRUNCATE) != 0;
  if (host_levels && truncate) return CDL_ERR_UNSUPPORTED;
  if (host_levels && chain_dtype != CDL_BF16) return CDL_ERR_UNSUPPORTED;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  if (chain_dtype != CDL_F64 && chain_dtype != CDL_F32 && chain_dtype != CDL_BF16 &&
      chain_dtype != CDL_FP8E4M3 && chain_dtype != CDL_FP8E4M3_T128)
    return CDL_ERR_INVALID_ARG;
  const bool fp8t = chain_dtype == CDL_FP8E4M3_T128;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A));
  CDL_TRY(dev_ptr(ctx, D));
  CDL_TRY(dev_ptr(ctx, vol));
  const bool tensor = chain_dtype == CDL_BF16 || chain_dtype == CDL_FP8E4M3 || fp8t;
  if (tensor && !tc_supported(ctx)) return CDL_ERR_UNSUPPORTED;
  const int64_t npad = round_up(n, 256);
  cdl_chain* ch = *inout;
  if (ch) {
    if (ch->n != n || ch->d != d || ch->dtype != chain_dtype || ch->device != ctx->device ||
        ch->host_levels != host_levels || (host_levels && ch->resident != std::min(resident, d)) || ch->regen)
      return CDL_ERR_INVALID_ARG;
  } else {
    ch = new cdl_chain();
    ch->device = ctx->device;
    ch->n = n;
    ch->npad = npad;
    ch->d = d;
    ch->dtype = chain_dtype;
    ch->elem = chain_dtype == CDL_F64 ? 8 : chain_dtype == CDL_F32 ? 4 : chain_dtype == CDL_BF16 ? 2 : 1;
    ch->resident = resident;
    size_t bytes = host_levels ? (2 + (size_t)std::min(resident, d)) * npad * npad * ch->elem
                               : (size_t)d * npad * npad * ch->elem;
    const size_t aop_bytes = tensor ? 2 * (size_t)npad * npad * 2 : 0;
    const size_t l16_bytes = (chain_dtype == CDL_FP8E4M3 || fp8t) ? (size_t)d * npad * npad * 2 : 0;
    const size_t ts_bytes = fp8t ? (size_t)d * (npad / 128) * (npad / 128) * sizeof(float) : 0;
    const size_t atom_bytes = fp8t ? 2 * (size_t)(npad / 128) * (npad / 128) * 512 : 0;
    // float-float residual operand (CUDA-core chains) or exact bf16 slices (tensor chains)
    const size_t ahl_bytes = tensor ? 0 : 2 * (size_t)n * n * sizeof(float);
    const size_t slice_bytes = tensor ? 6 * (size_t)npad * npad * 2 : 0;
    if (ctx->ws_cap && ctx->ws_used + bytes + aop_bytes + l16_bytes + ahl_bytes + slice_bytes > ctx->ws_cap) {
      delete ch;
      return CDL_ERR_OOM;
    }
    if ((ahl_bytes && cudaMalloc(&ch->ahl, ahl_bytes) != cudaSuccess) ||
        (slice_bytes && (cudaMalloc(&ch->aslices, slice_bytes) != cudaSuccess ||
                         cudaMalloc(&ch->a_scale, 2 * sizeof(double)) != cudaSuccess)) ||
        (aop_bytes && cudaMalloc(&ch->aop, aop_bytes) != cudaSuccess) ||
        (l16_bytes && (cudaMalloc(&ch->levels16, l16_bytes) != cudaSuccess ||
                       cudaMalloc(&ch->amax, d * sizeof(unsigned)) != cudaSuccess)) ||
        (ts_bytes && cudaMalloc(&ch->tscale, ts_bytes) != cudaSuccess) ||
        (atom_bytes && cudaMalloc(&ch->tatoms, atom_bytes) != cudaSuccess) ||
        (host_levels ? ooc_init(ch) != CDL_OK : cudaMalloc(&ch->levels, bytes) != cudaSuccess) ||
        cudaMalloc(&ch->rsqrt_d, npad * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ch->D, npad * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ch->vol, sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      cdl_chain_free(ch);
      return CDL_ERR_OOM;
    }
  }
  CDL_CUDA_TRY(cudaMemcpyAsync(ch->D, D, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if (npad > n)
    CDL_CUDA_TRY(cudaMemsetAsync(ch->D + n, 0, (npad - n) * sizeof(double), ctx->stream));
  CDL_CUDA_TRY(cudaMemcpyAsync(ch->vol, vol, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  int st = chain_init(ctx, ch, static_cast<const double*>(A));
  ch->d_eff = d;
  unsigned* norm_bits = nullptr;
  if (truncate) {
    void* vn;
    st = st == CDL_OK ? ws_get(ctx, "chain.norm", sizeof(unsigned), &vn) : st;
    norm_bits = static_cast<unsigned*>(vn);
  }
  for (int i = 0; st == CDL_OK && i + 1 < d; ++i) {
    if (chain_dtype == CDL_FP8E4M3) st = fp8_level_bound(ctx, ch, i);
    if (st == CDL_OK)
      st = fp8t ? chain_square_fp8t(ctx, ch, i) : tensor ? chain_square_tc(ctx, ch, i) : chain_square_simt(ctx, ch, i);
    if (st == CDL_OK && truncate) {
      // ||S~_{i+1}||_2 <= its max row sum; at 2^-24 or less neither it nor the
      // levels after it (their norms square) can change a float32 x + S~ x
      st = level_inf_norm(ctx, ch, i + 1, norm_bits);
      unsigned bits = 0;
      if (st == CDL_OK) st = cudaMemcpyAsync(&bits, norm_bits, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream)
                                 == cudaSuccess ? CDL_OK : CDL_ERR_CUDA;
      if (st == CDL_OK) st = cudaStreamSynchronize(ctx->stream) == cudaSuccess ? CDL_OK : CDL_ERR_CUDA;
      float eta;
      std::memcpy(&eta, &bits, sizeof(float));
      if (st == CDL_OK && eta <= 0x1p-24f) {
        ch->d_eff = i + 1;
        break;
      }
    }
  }
  if (st != CDL_OK) {
    if (!*inout) cdl_chain_free(ch);
    return st;
  }
  *inout = ch;
  return CDL_OK;
}

int cdl_project(cdl_ctx* ctx, const void* A, cdl_dtype a_dtype, int64_t n, int32_t k,
                uint64_t seed, double* Y) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || k < 1 || k > 1024) return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A));
  CDL_TRY(dev_ptr(ctx, Y));
  return project(ctx, static_cast<const double*>(A), n, k, seed, Y);
}

int cdl_chain_solve(cdl_ctx* ctx, const cdl_chain* ch, const void* A, cdl_dtype a_dtype,
                    const double* Y, int32_t k, const cdl_solve_opts* opts, double* Z,
                    cdl_solve_stats* stats) {
  if (!ctx || !ch || !opts) return CDL_ERR_INVALID_ARG;
  if (k < 1 || k > 1024 || opts->max_iter < 1 || opts->rel_tol < 0 ||
      (opts->flags & ~CDL_SOLVE_FULL_RESIDUAL) != 0)
    return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  if (ch->device != ctx->device) return CDL_ERR_INVALID_ARG;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A));
  CDL_TRY(dev_ptr(ctx, Y));
  CDL_TRY(dev_ptr(ctx, Z));
  return chain_solve(ctx, ch, static_cast<const double*>(A), Y, k, opts, Z, stats);
}

int cdl_cad_score(cdl_ctx* ctx, const void* A1, const void* A2, cdl_dtype a_dtype,
                  const double* Z1, const double* Z2, const double* vol1, const double* vol2,
                  int64_t n, int32_t k, cdl_dtype score_dtype, int32_t topk, double* F,
                  int64_t* top_idx) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  if (score_dtype != CDL_F64 && score_dtype != CDL_F32 && score_dtype != CDL_BF16) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || k < 1 || k > 1024 || topk < 0 || topk > 1024 || topk > n)
    return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A1));
  CDL_TRY(dev_ptr(ctx, A2));
  CDL_TRY(dev_ptr(ctx, Z1));
  CDL_TRY(dev_ptr(ctx, Z2));
  CDL_TRY(dev_ptr(ctx, vol1));
  CDL_TRY(dev_ptr(ctx, vol2));
  CDL_TRY(dev_ptr(ctx, F));
  if (topk > 0) CDL_TRY(dev_ptr(ctx, top_idx));
  return cad_score(ctx, static_cast<const double*>(A1), static_cast<const double*>(A2), Z1, Z2,
                   vol1, vol2, n, k, score_dtype, topk, F, top_idx);
}

int cdl_cad_edges(cdl_ctx* ctx, const void* A1, const void* A2, cdl_dtype a_dtype, const double* Z1, const double* Z2,
                  const double* vol1, const double* vol2, int64_t n, int32_t k, cdl_dtype score_dtype, double delta,
                  int64_t max_edges, int64_t* edge_ij, double* edge_dE, const int64_t* nodes, int32_t n_nodes,
                  int32_t top_per_node, int64_t* partner, double* partner_dE, double* F, cdl_edge_result* res) {
  if (!ctx || !res) return CDL_ERR_INVALID_ARG;
  if (score_dtype != CDL_F64 && score_dtype != CDL_F32) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > 65536 || k < 1 || k > 1024 || !(delta > 0) || max_edges < 0 || n_nodes < 0 ||
      n_nodes > 65535 || top_per_node < 0 || top_per_node > 1024)
    return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A1));
  CDL_TRY(dev_ptr(ctx, A2));
  CDL_TRY(dev_ptr(ctx, Z1));
  CDL_TRY(dev_ptr(ctx, Z2));
  CDL_TRY(dev_ptr(ctx, vol1));
  CDL_TRY(dev_ptr(ctx, vol2));
  if (max_edges > 0) {
    CDL_TRY(dev_ptr(ctx, edge_ij));
    CDL_TRY(dev_ptr(ctx, edge_dE));
  }
  if (n_nodes > 0 && top_per_node > 0) {
    CDL_TRY(dev_ptr(ctx, nodes));
    CDL_TRY(dev_ptr(ctx, partner));
    CDL_TRY(dev_ptr(ctx, partner_dE));
  }
  if (F) CDL_TRY(dev_ptr(ctx, F));
  return cad_edges(ctx, static_cast<const double*>(A1), static_cast<const double*>(A2), Z1, Z2, vol1, vol2, n, k,
                   score_dtype == CDL_F64, delta, max_edges, nodes, n_nodes, top_per_node, edge_ij, edge_dE, partner,
                   partner_dE, F, res);
}

int cdl_changed_nodes(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n, int32_t T, int32_t* changed,
                      int32_t* n_changed) {
  if (!ctx || !n_changed) return CDL_ERR_INVALID_ARG;
  if (n < 1 || n > (1 << 20) || T < 1 || T > 4096) return CDL_ERR_INVALID_ARG;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, X1));
  CDL_TRY(dev_ptr(ctx, X2));
  CDL_TRY(dev_ptr(ctx, changed, 4));
  void* vc;
  CDL_TRY(ws_get(ctx, "score.changed_count", sizeof(int), &vc));
  CDL_TRY(changed_nodes(ctx, X1, X2, n, T, changed, static_cast<int*>(vc)));
  CDL_CUDA_TRY(cudaMemcpyAsync(n_changed, vc, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return CDL_OK;
}

int cdl_cad_score_changed(cdl_ctx* ctx, const void* A1, const void* A2, cdl_dtype a_dtype, const double* Z1,
                          const double* Z2, const double* vol1, const double* vol2, int64_t n, int32_t k,
                          cdl_dtype score_dtype, const int32_t* changed, int32_t n_changed, int32_t topk,
                          double* F, int64_t* top_idx) {
  if (!ctx) return CDL_ERR_INVALID_ARG;
  if (score_dtype != CDL_F64 && score_dtype != CDL_F32) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || k < 1 || k > 1024 || topk < 0 || topk > 1024 || topk > n || n_changed < 0 ||
      n_changed > n || n_changed > 65535)
    return CDL_ERR_INVALID_ARG;
  if (a_dtype != CDL_F64) return CDL_ERR_UNSUPPORTED;
  CDL_TRY(set_device(ctx));
  CDL_TRY(dev_ptr(ctx, A1));
  CDL_TRY(dev_ptr(ctx, A2));
  CDL_TRY(dev_ptr(ctx, Z1));
  CDL_TRY(dev_ptr(ctx, Z2));
  CDL_TRY(dev_ptr(ctx, vol1));
  CDL_TRY(dev_ptr(ctx, vol2));
  CDL_TRY(dev_ptr(ctx, F));
  if (n_changed > 0) CDL_TRY(dev_ptr(ctx, changed, 4));
  if (topk > 0) CDL_TRY(dev_ptr(ctx, top_idx));
  return cad_score_changed(ctx, static_cast<const double*>(A1), static_cast<const double*>(A2), Z1, Z2, vol1, vol2,
                           n, k, score_dtype == CDL_F64, changed, n_changed, topk, F, top_idx);
}

int cdl_caddelag_pair(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n, int32_t T,
                      const cdl_pair_opts* o, double* F, int64_t* top_idx,
                      cdl_solve_stats* stats1, cdl_solve_stats* stats2) {
  if (!ctx || !o || !X1 || !X2 || !F) return CDL_ERR_INVALID_ARG;
  if (n < 2 || n > (1 << 20) || T < 1 || T > 4096 || o->k < 1 || o->k > 1024 || o->d < 1 ||
      o->topk < 0 || o->topk > 1024 || o->topk > n || (o->topk > 0 && !top_idx) ||
      (o->score_dtype != CDL_F64 && o->score_dtype != CDL_F32 && o->score_dtype != CDL_BF16) ||
      (o->score_flags & ~CDL_SCORE_CHANGED_ONLY) ||
      ((o->score_flags & CDL_SCORE_CHANGED_ONLY) && (!(o->sigma > 0) || o->score_dtype == CDL_BF16)) ||
      (o->chain_flags & ~(CDL_CHAIN_HOST_LEVELS | CDL_CHAIN_TRUNCATE | CDL_CHAIN_RESIDENT_MASK |
                          CDL_PAIR_REGEN_GRAPHS | CDL_PAIR_PANEL_MASK)))
    return CDL_ERR_INVALID_ARG;
  CDL_TRY(set_device(ctx));
  if (o->chain_flags & CDL_PAIR_REGEN_GRAPHS) {
    if (o->chain_flags & CDL_CHAIN_TRUNCATE) return CDL_ERR_UNSUPPORTED;
    return pair_regen(ctx, X1, X2, n, T, o, F, top_idx, stats1, stats2);
  }
  if (o->chain_flags & CDL_PAIR_PANEL_MASK) return CDL_ERR_INVALID_ARG;
  const size_t nn = (size_t)n * n;
  void *dX, *dA1, *dA2, *dvec, *dY, *dZ1, *dZ2, *dF, *dtop;
  CDL_TRY(ws_get(ctx, "pair.X", 2 * (size_t)n * T * sizeof(double), &dX));
  CDL_TRY(ws_get(ctx, "pair.A1", nn * sizeof(double), &dA1));
  CDL_TRY(ws_get(ctx, "pair.A2", nn * sizeof(double), &dA2));
  CDL_TRY(ws_get(ctx, "pair.vec", (2 * (size_t)n + 8) * sizeof(double), &dvec));
  CDL_TRY(ws_get(ctx, "pair.Y", (size_t)n * o->k * sizeof(double), &dY));
  CDL_TRY(ws_get(ctx, "pair.Z1", (size_t)n * o->k * sizeof(double), &dZ1));
  CDL_TRY(ws_get(ctx, "pair.Z2", (size_t)n * o->k * sizeof(double), &dZ2));
  CDL_TRY(ws_get(ctx, "pair.F", (size_t)n * sizeof(double), &dF));
  CDL_TRY(ws_get(ctx, "pair.top", (size_t)(o->topk + 1) * sizeof(int64_t), &dtop));
  double* x1 = static_cast<double*>(dX);
  double* x2 = x1 + (size_t)n * T;
  if (o->host_io) {
    CDL_CUDA_TRY(cudaMemcpyAsync(x1, X1, (size_t)n * T * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CDL_CUDA_TRY(cudaMemcpyAsync(x2, X2, (size_t)n * T * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  } else {
    x1 = const_cast<double*>(X1);
    x2 = const_cast<double*>(X2);
    CDL_TRY(dev_ptr(ctx, X1));
    CDL_TRY(dev_ptr(ctx, X2));
  }
  double* D1 = static_cast<double*>(dvec);
  double* D2 = D1 + n;
  double* sc = D2 + n;   // vol1, vol2, sigma1, sigma2
  double* Zs[2] = {static_cast<double*>(dZ1), static_cast<double*>(dZ2)};
  double* As[2] = {static_cast<double*>(dA1), static_cast<double*>(dA2)};
  double* Ds[2] = {D1, D2};
  const double* Xs[2] = {x1, x2};
  cdl_solve_stats* sts[2] = {stats1, stats2};
  if (ctx->pair_chain && (ctx->pair_chain->n != n || ctx->pair_chain->d != o->d ||
                          ctx->pair_chain->dtype != o->chain_dtype ||
                          ctx->pair_chain->host_levels != ((o->chain_flags & CDL_CHAIN_HOST_LEVELS) != 0) ||
                          ctx->pair_chain->resident !=
                              std::min(o->d, (o->chain_flags & CDL_CHAIN_RESIDENT_MASK) >> CDL_CHAIN_RESIDENT_SHIFT))) {
    CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cdl_chain_free(ctx->pair_chain);
    ctx->pair_chain = nullptr;
  }
  bool converged = true;
  void* vamax;
  CDL_TRY(ws_get(ctx, "pair.amax", sizeof(unsigned long long), &vamax));
  unsigned long long* amax = static_cast<unsigned long long*>(vamax);
  for (int g = 0; g < 2; ++g) {
    CDL_TRY(graph_build(ctx, Xs[g], n, T, o->sigma, As[g], Ds[g], sc + g, sc + 2 + g, 0, amax));
    ctx->amax_hint_A = As[g];   // the chain build takes max A from the graph build
    ctx->amax_hint_bits = amax;
    const int cst = cdl_chain_build(ctx, As[g], CDL_F64, Ds[g], sc + g, n, o->d, o->chain_dtype, o->chain_flags,
                                    &ctx->pair_chain);
    ctx->amax_hint_A = nullptr;
    ctx->amax_hint_bits = nullptr;
    CDL_TRY(cst);
    // tensor chains hold the float64 bits of max |A| (found by their build): the
    // projection reuses them instead of another pass over A
    const cdl_chain* pc = ctx->pair_chain;
    CDL_TRY(project(ctx, As[g], n, o->k, o->seed, static_cast<double*>(dY),
                    pc->a_scale ? reinterpret_cast<const unsigned long long*>(pc->a_scale + 1) : nullptr));
    int st = chain_solve(ctx, ctx->pair_chain, As[g], static_cast<double*>(dY), o->k, &o->solve,
                         Zs[g], sts[g]);
    if (st != CDL_OK && st != CDL_ERR_NOT_CONVERGED) return st;
    converged = converged && st == CDL_OK;
  }
  double* Fd = o->host_io ? static_cast<double*>(dF) : F;
  int64_t* topd = o->host_io ? static_cast<int64_t*>(dtop) : top_idx;
  if (o->score_flags & CDL_SCORE_CHANGED_ONLY) {
    // shared sigma: only edges of nodes whose series changed have Delta A != 0
    void *vlist, *vcount;
    CDL_TRY(ws_get(ctx, "pair.changed", (size_t)n * sizeof(int), &vlist));
    CDL_TRY(ws_get(ctx, "pair.changed_count", sizeof(int), &vcount));
    CDL_TRY(changed_nodes(ctx, x1, x2, n, T, static_cast<int*>(vlist), static_cast<int*>(vcount)));
    int m = 0;
    CDL_CUDA_TRY(cudaMemcpyAsync(&m, vcount, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (m > 65535) return CDL_ERR_UNSUPPORTED;
    CDL_TRY(cad_score_changed(ctx, As[0], As[1], Zs[0], Zs[1], sc, sc + 1, n, o->k, o->score_dtype == CDL_F64,
                              static_cast<const int*>(vlist), m, o->topk, Fd, topd));
  } else {
    CDL_TRY(cad_score(ctx, As[0], As[1], Zs[0], Zs[1], sc, sc + 1, n, o->k, o->score_dtype, o->topk, Fd, topd));
  }
  ctx->last_pair.n = n;
  ctx->last_pair.k = o->k;
  for (int g = 0; g < 2; ++g) {
    ctx->last_pair.Z[g] = Zs[g];
    ctx->last_pair.vol[g] = sc + g;
    ctx->last_pair.sigma[g] = sc + 2 + g;
  }
  if (o->host_io) {
    CDL_CUDA_TRY(cudaMemcpyAsync(F, Fd, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (o->topk > 0)
      CDL_CUDA_TRY(cudaMemcpyAsync(top_idx, topd, (size_t)o->topk * sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  return converged ? CDL_OK : CDL_ERR_NOT_CONVERGED;
}

int cdl_pair_embeddings(cdl_ctx* ctx, double* Z1, double* Z2, double* scalars) {
  if (!ctx || !ctx->last_pair.Z[0]) return CDL_ERR_INVALID_ARG;
  CDL_TRY(set_device(ctx));
  const size_t nk = (size_t)ctx->last_pair.n * ctx->last_pair.k;
  double* Zo[2] = {Z1, Z2};
  for (int g = 0; g < 2; ++g)
    if (Zo[g]) CDL_CUDA_TRY(cudaMemcpyAsync(Zo[g], ctx->last_pair.Z[g], nk * sizeof(double), cudaMemcpyDefault,
                                            ctx->stream));
  if (scalars) {
    const double* src[4] = {ctx->last_pair.vol[0], ctx->last_pair.vol[1], ctx->last_pair.sigma[0],
                            ctx->last_pair.sigma[1]};
    for (int q = 0; q < 4; ++q)
      CDL_CUDA_TRY(cudaMemcpyAsync(scalars + q, src[q], sizeof(double), cudaMemcpyDefault, ctx->stream));
  }
  CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return CDL_OK;
}

}  // extern "C"
