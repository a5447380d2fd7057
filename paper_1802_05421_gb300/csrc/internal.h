// Library-internal declarations shared by the translation units of libcdl.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "cdl.h"

#define CDL_TRY(expr)                         \
  do {                                        \
    int _st = (expr);                         \
    if (_st != CDL_OK) return _st;            \
  } while (0)

#define CDL_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      cdl::set_last_error(cudaGetErrorString(_e), __FILE__, __LINE__);            \
      return CDL_ERR_CUDA;                                                        \
    }                                                                             \
  } while (0)

namespace cdl {

void set_last_error(const char* msg, const char* file, int line);

// Device-side status word: kernels with bounded waits write a nonzero code
// here when a wait expires (they then return early instead of hanging).
enum : unsigned { DEV_OK = 0u, DEV_WAIT_TIMEOUT = 1u };

struct Event2 {
  cudaEvent_t a = nullptr, b = nullptr;
  int kc = 0;
  double work = 0.0;
};

}  // namespace cdl

struct cdl_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t ws_cap = 0;
  size_t ws_used = 0;
  int sm_count = 0;
  // grow-only named workspace buffers
  std::map<std::string, std::pair<void*, size_t>> ws;
  // device status word (bounded-wait expiry), 4 bytes
  unsigned* dev_status = nullptr;
  // launch accounting
  int64_t launches = 0;
  bool timing = false;
  std::vector<cdl::Event2> pending;   // recorded, not yet folded into totals
  std::vector<cudaEvent_t> free_events;
  double kc_ms[CDL_KC_COUNT] = {0};
  int64_t kc_launches[CDL_KC_COUNT] = {0};
  double kc_work[CDL_KC_COUNT] = {0};
  // chains owned by cdl_caddelag_pair
  cdl_chain* pair_chain = nullptr;
  // tile schedules uploaded to the workspace, by workspace name -> tile count
  std::map<std::string, int> tile_lists;
  int debug_flags = 0;   // CDL_DEBUG_* test hooks
};

struct cdl_chain {
  int device = 0;
  int64_t n = 0, npad = 0;
  int32_t d = 0;
  cdl_dtype dtype = CDL_F64;
  size_t elem = 8;
  void* levels = nullptr;     // d * npad * npad elements
  void* aop = nullptr;        // bf16 chains: A = A_hi + A_lo as two bf16 npad x npad matrices
  void* levels16 = nullptr;   // fp8 chains: bf16 copies of the levels (the apply's operand)
  unsigned* amax = nullptr;   // fp8 chains: per-level bound of |value| (float bits), scale = amax/448
  float* ahl = nullptr;       // A as float hi + lo planes (n x n each), the float-float residual's operand
  double* rsqrt_d = nullptr;  // npad: D_i^{-1/2} (0 in padding)
  double* D = nullptr;        // npad: degrees (0 in padding)
  double* vol = nullptr;      // 1
  void* level(int i) const {
    return static_cast<char*>(levels) + (size_t)i * (size_t)npad * (size_t)npad * elem;
  }
  // bf16 view of level i used by the apply (the level itself for bf16 chains)
  void* level16(int i) const {
    if (!levels16) return level(i);
    return static_cast<char*>(levels16) + (size_t)i * (size_t)npad * (size_t)npad * 2;
  }
};

namespace cdl {

// Workspace: returns a device buffer of at least `bytes` for `name`,
// reusing or growing it (respecting ctx->ws_cap).
int ws_get(cdl_ctx* ctx, const char* name, size_t bytes, void** out);

// Launch accounting: call before and after each kernel launch.
struct Launch {
  cdl_ctx* ctx;
  int kc;
  double work;
  cudaEvent_t a = nullptr;
  Launch(cdl_ctx* c, int k, double w);
  int done();   // checks cudaGetLastError, records the end event
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---- kernel launchers (one per translation unit family) ----
// graph.cu
int graph_build(cdl_ctx* ctx, const double* X, int64_t n, int T, double sigma, double* A,
                double* D, double* vol, double* sigma_out);
int graph_build_static(const double* X, int64_t n, int T, double sigma, double* A, double* D,
                       double* vol, double* sigma_out, cudaStream_t stream);
// chain.cu
int chain_init(cdl_ctx* ctx, cdl_chain* ch, const double* A);
int chain_square_simt(cdl_ctx* ctx, cdl_chain* ch, int level);
int fp8_level_bound(cdl_ctx* ctx, cdl_chain* ch, int level);
int apply_simt(cdl_ctx* ctx, const cdl_chain* ch, int level, const void* x, void* partial,
               int k, int splits);
// tc_gemm.cu
int chain_square_tc(cdl_ctx* ctx, cdl_chain* ch, int level);
int apply_tc(cdl_ctx* ctx, const cdl_chain* ch, int level, const void* xop, float* partial,
             int k, int splits);
int apply_tc_mat(cdl_ctx* ctx, const void* amat, int np, const void* xop, float* partial, int kp,
                 int splits);
bool tc_supported(cdl_ctx* ctx);
// solve.cu
int chain_solve(cdl_ctx* ctx, const cdl_chain* ch, const double* A, const double* Y, int k,
                const cdl_solve_opts* opts, double* Z, cdl_solve_stats* stats);
// project.cu
int project(cdl_ctx* ctx, const double* A, int64_t n, int k, uint64_t seed, double* Y);
// score.cu
int cad_score(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1,
              const double* Z2, const double* vol1, const double* vol2, int64_t n, int k,
              bool fp64, int topk, double* F, int64_t* top_idx);

}  // namespace cdl
