// Alg. 4 for one graph pair whose dense graphs are not kept: each graph is
// regenerated from its node series in row panels of P rows wherever it is
// needed (the paper's larger-than-memory aim, Sec. 1 and Sec. 3.2: there the
// block matrices live on a shared file system; here one GPU recomputes row
// blocks of A from the n x T series instead of storing n^2 values):
//
//   sigma  the exact lower median by radix select, each histogram pass over
//          the upper-triangle part of every panel's exact squared distances;
//   D, vol the panels' row sums;
//   chain  level-0 rows from each panel, then the d - 1 squarings (bf16,
//          tcgen05), levels 0 .. resident - 1 in device memory and the rest
//          in pinned host memory (CDL_CHAIN_HOST_LEVELS);
//   Y      the projection's rows from the same panels (Alg. 1 / Alg. 3);
//   solve  Richardson refinement with the full float64-class residual every
//          step, A Z summed over the panels' transposed exact slices;
//   scores both graphs' panels together, the score tiles of the panel's rows.
//
// Panel A values equal the ones cdl_build_graph stores (exact distances, the
// same exponential); degrees and sums differ only in summation order.
#include <algorithm>

#include "internal.h"

namespace cdl {

namespace {

int resident_levels(cdl_ctx* ctx, int64_t npad, int d, int requested, size_t reserve) {
  if (requested != 255) return std::min(requested, d);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t lb = (size_t)npad * npad * 2;
  const size_t slots = 2 * lb;
  if (free_b < slots + reserve) return 0;
  return (int)std::min<size_t>((size_t)d, (free_b - slots - reserve) / lb);
}

}  // namespace

int pair_regen(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n64, int T, const cdl_pair_opts* o,
               double* F, int64_t* top_idx, cdl_solve_stats* stats1, cdl_solve_stats* stats2) {
  if (o->chain_dtype != CDL_BF16 || o->score_dtype != CDL_BF16 || o->score_flags != 0)
    return CDL_ERR_UNSUPPORTED;
  const int n = (int)n64;
  const int k = o->k;
  const int plog = (o->chain_flags & CDL_PAIR_PANEL_MASK) >> CDL_PAIR_PANEL_SHIFT;
  if (plog && (plog < 8 || plog > 16)) return CDL_ERR_INVALID_ARG;
  const int64_t npad = round_up(n64, 256);
  const int P = (int)std::min<int64_t>(plog ? (1 << plog) : 4096, npad);   // a multiple of 256
  const bool host_levels = (o->chain_flags & CDL_CHAIN_HOST_LEVELS) != 0;
  const int res_req = host_levels ? (o->chain_flags & CDL_CHAIN_RESIDENT_MASK) >> CDL_CHAIN_RESIDENT_SHIFT : o->d;
  cudaStream_t s = ctx->stream;

  // buffers: two float64 panels, the transposed slices of one, the series,
  // degrees, scalars, Y, Z1, Z2, F, top
  void *dP, *dS, *dX, *dvec, *dY, *dZ1, *dZ2, *dF, *dtop;
  CDL_TRY(ws_get(ctx, "regen.panels", 2 * (size_t)P * n * sizeof(double), &dP));
  CDL_TRY(ws_get(ctx, "regen.slicesT", 6 * (size_t)npad * P * 2, &dS));
  CDL_TRY(ws_get(ctx, "regen.vec", (3 * (size_t)n + 8) * sizeof(double), &dvec));
  CDL_TRY(ws_get(ctx, "regen.Y", (size_t)n * k * sizeof(double), &dY));
  CDL_TRY(ws_get(ctx, "regen.Z1", (size_t)n * k * sizeof(double), &dZ1));
  CDL_TRY(ws_get(ctx, "regen.Z2", (size_t)n * k * sizeof(double), &dZ2));
  CDL_TRY(ws_get(ctx, "regen.F", (size_t)n * sizeof(double), &dF));
  CDL_TRY(ws_get(ctx, "regen.top", (size_t)(o->topk + 1) * sizeof(int64_t), &dtop));
  double* panel[2] = {static_cast<double*>(dP), static_cast<double*>(dP) + (size_t)P * n};
  const double* Xs[2] = {X1, X2};
  if (o->host_io) {
    CDL_TRY(ws_get(ctx, "regen.X", 2 * (size_t)n * T * sizeof(double), &dX));
    double* x = static_cast<double*>(dX);
    CDL_CUDA_TRY(cudaMemcpyAsync(x, X1, (size_t)n * T * sizeof(double), cudaMemcpyHostToDevice, s));
    CDL_CUDA_TRY(cudaMemcpyAsync(x + (size_t)n * T, X2, (size_t)n * T * sizeof(double), cudaMemcpyHostToDevice, s));
    Xs[0] = x;
    Xs[1] = x + (size_t)n * T;
  } else {
    CDL_TRY(check_dev_ptr(ctx, X1, 8));
    CDL_TRY(check_dev_ptr(ctx, X2, 8));
  }
  double* D1 = static_cast<double*>(dvec);
  double* D2 = D1 + n;
  double* Dscr = D2 + n;
  double* sc = Dscr + n;   // vol1, vol2
  double* Zs[2] = {static_cast<double*>(dZ1), static_cast<double*>(dZ2)};
  double* Ds[2] = {D1, D2};
  cdl_solve_stats* sts[2] = {stats1, stats2};
  RegenGraph G[2];

  // the chain: one for both graphs (rebuilt in place), kept by the context
  const bool keep_ok = ctx->regen_chain && ctx->regen_chain->n == n64 && ctx->regen_chain->d == o->d &&
                       (host_levels ? (res_req == 255 || ctx->regen_chain->resident == std::min(res_req, o->d))
                                    : ctx->regen_chain->resident == o->d);
  if (ctx->regen_chain && !keep_ok) {
    CDL_CUDA_TRY(cudaStreamSynchronize(s));
    cdl_chain_free(ctx->regen_chain);
    ctx->regen_chain = nullptr;
  }
  if (!ctx->regen_chain) {
    const size_t reserve = (size_t)24 << 30;   // the rest of this call's buffers and headroom
    const int resident = host_levels ? resident_levels(ctx, npad, o->d, res_req, reserve) : o->d;
    CDL_TRY(chain_create_regen(ctx, n64, o->d, resident, &ctx->regen_chain));
  }
  cdl_chain* ch = ctx->regen_chain;
  if (ch->resident < 1) return CDL_ERR_UNSUPPORTED;   // level 0 is formed in place, panel by panel

  unsigned long long* one_bits = reinterpret_cast<unsigned long long*>(ch->a_scale + 1);   // max A <= 1
  bool converged = true;
  for (int g = 0; g < 2; ++g) {
    G[g].id = g;
    G[g].D = Ds[g];
    G[g].vol = sc + g;
    CDL_TRY(graph_regen_init(ctx, G[g], Xs[g], n64, T, o->sigma, panel[0], P));
    // chain vectors from this graph's degrees, then level 0 and Y from the same panels
    CDL_CUDA_TRY(cudaMemcpyAsync(ch->D, Ds[g], (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (npad > n) CDL_CUDA_TRY(cudaMemsetAsync(ch->D + n, 0, (size_t)(npad - n) * sizeof(double), s));
    CDL_CUDA_TRY(cudaMemcpyAsync(ch->vol, sc + g, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CDL_TRY(chain_vectors_only(ctx, ch));
    void* L0 = ooc_write_begin(ctx, ch, 0);
    if (npad > n)   // padding rows of level 0
      CDL_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(L0) + (size_t)n * npad * 2, 0, (size_t)(npad - n) * npad * 2, s));
    for (int r0 = 0; r0 < n; r0 += P) {
      const int rows = std::min(P, n - r0);
      CDL_TRY(regen_panel(ctx, G[g], panel[0], r0, rows, Dscr));
      CDL_TRY(chain_level0_panel(ctx, ch, L0, panel[0], r0, rows));
      CDL_TRY(project_panel(ctx, panel[0], n64, r0, rows, k, o->seed, static_cast<double*>(dY), one_bits));
    }
    CDL_TRY(ooc_write_end(ctx, ch, 0));
    CDL_TRY(project_center(ctx, n64, k, static_cast<double*>(dY)));
    for (int i = 0; i + 1 < o->d; ++i) CDL_TRY(chain_square_tc(ctx, ch, i));
    RegenSource src;
    src.g = &G[g];
    src.panel = panel[0];
    src.slicesT = dS;
    src.Dscratch = Dscr;
    src.P = P;
    ch->regen = &src;
    const int st = chain_solve(ctx, ch, nullptr, static_cast<double*>(dY), k, &o->solve, Zs[g], sts[g]);
    ch->regen = nullptr;
    if (st == CDL_ERR_NOT_CONVERGED)
      converged = false;
    else
      CDL_TRY(st);
  }
  // scores: rows r0 .. of both graphs regenerated side by side
  auto fill = [&](int r0, int rows, const double** a1, const double** a2) -> int {
    CDL_TRY(regen_panel(ctx, G[0], panel[0], r0, rows, Dscr));
    CDL_TRY(regen_panel(ctx, G[1], panel[1], r0, rows, Dscr));
    *a1 = panel[0];
    *a2 = panel[1];
    return CDL_OK;
  };
  double* Fo = o->host_io ? static_cast<double*>(dF) : F;
  int64_t* To = o->host_io ? static_cast<int64_t*>(dtop) : top_idx;
  if (!o->host_io) {
    CDL_TRY(check_dev_ptr(ctx, F, 8));
    if (o->topk > 0) CDL_TRY(check_dev_ptr(ctx, top_idx, 8));
  }
  CDL_TRY(cad_score_panels(ctx, Zs[0], Zs[1], sc, sc + 1, n64, k, P, fill, o->topk, Fo, To));
  ctx->last_pair.n = n64;
  ctx->last_pair.k = k;
  for (int g = 0; g < 2; ++g) {
    ctx->last_pair.Z[g] = Zs[g];
    ctx->last_pair.vol[g] = sc + g;
    ctx->last_pair.sigma[g] = G[g].sigma;
  }
  if (o->host_io) {
    CDL_CUDA_TRY(cudaMemcpyAsync(F, Fo, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (o->topk > 0)
      CDL_CUDA_TRY(cudaMemcpyAsync(top_idx, To, (size_t)o->topk * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CDL_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return converged ? CDL_OK : CDL_ERR_NOT_CONVERGED;
}

}  // namespace cdl
