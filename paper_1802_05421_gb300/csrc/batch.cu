// Batched form: many independent graph pairs of uneven order embedded and
// scored together (Alg. 4 for each pair; the k right-hand sides of each graph
// run together as in Sec. 4.1, and here the graphs of the batch do too).
//
// A plan, built on the first call for a given set of sizes and options, owns
// every device buffer of the batch in one allocation, the per-graph tensor
// maps of the grouped tcgen05 launches, the tile tables of the grouped
// kernels and a private context (own stream and workspace). Each chain
// level is squared for all graphs in one grouped launch, each refinement step
// runs as one launch per kernel over all graphs (graphs that have converged
// skip their tiles), and the scores of all pairs come from one grouped
// launch per scoring step. The refinement runs a fixed number of steps on the
// host side and decides per graph on the device, so a whole call has no
// host synchronisation and can be recorded once as a CUDA graph and
// replayed.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace cdl {

struct BatchPlan {
  // key
  int G = 0, T = 0, k = 0, d = 0, topk = 0, score_dtype = 0;
  std::vector<int64_t> n;
  uint64_t seed = 0;
  double sigma = 0;
  cdl_solve_opts solve{};
  // resources
  cdl_ctx* inner = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr;
  void* mem = nullptr;
  size_t bytes = 0;
  int64_t N = 0;                 // total nodes over the pairs
  std::vector<int64_t> off;      // first row of pair p
  std::vector<cdl_chain> chains; // views into mem
  std::vector<double*> A, Dv, scal, Y;
  double* X = nullptr;           // 2N x T: first graphs, then second graphs
  double* F = nullptr;           // N
  int64_t* top = nullptr;        // G x topk
  std::vector<int> order;        // graphs by order, largest first
  BatchSolve bs;
  GraphBatch gb;
  const PGraph* pgs = nullptr;
  // level 0 of every graph in three grouped launches
  const CGraph* cgs = nullptr;
  BTiles cvec, cinit;
  double cinit_bytes = 0;
  // autotuned variants: squaring tile width per graph size, projection rows per block
  struct SqVariant {
    int max_npad_128;            // graphs up to this order use 128 x 128 tiles; -1: CTA pairs (256 x 256)
    std::vector<TcGroup> first;  // host copy of entry 0 of each level's array
    TcGroup* groups = nullptr;   // device, (d - 1) x G2
    BTiles tiles;
    double ms = 0;
  };
  struct ProjVariant {
    int rpb;
    BTiles blocks;
    double ms = 0;
  };
  std::vector<SqVariant> sqv;
  std::vector<ProjVariant> pv;
  int sq_choice = 0, pv_choice = 0;
  bool tuned = false;
  double proj_adds = 0;
  std::vector<TcGroup> lvl_first, res_first;
  BTiles score_elem, score_pairs, score_nodes;
  ScoreJob* jobs = nullptr;
  unsigned* cmax = nullptr;      // G x 2k column bounds of the float32 scoring
  std::vector<BState> st_host;
  double sq_flops = 0, score_bytes = 0;
  int* active = nullptr;         // device: graphs still refining after the last slot
  int slots_seen = 0;            // most slots a call has needed so far
  int slots_captured = 0;        // slots recorded in the CUDA graph
  cudaGraphExec_t exec = nullptr;
  int64_t graph_launches = 0;
  int64_t graph_kc_launches[CDL_KC_COUNT] = {0};
  double graph_kc_work[CDL_KC_COUNT] = {0};
};

void batch_plan_free(BatchPlan* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->inner) cdl_ctx_destroy(p->inner);
  if (p->mem) cudaFree(p->mem);
  if (p->ev_in) cudaEventDestroy(p->ev_in);
  if (p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

namespace {

// Bump allocator over one device block: a sizing pass (base == nullptr),
// then an assigning pass.
struct Carver {
  char* base = nullptr;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += std::max<size_t>(count * sizeof(T), 1);
    return p;
  }
};

bool same_key(const BatchPlan* p, int G, const int64_t* n, int T, const cdl_batch_opts* o) {
  if (!p || p->G != G || p->T != T || p->k != o->k || p->d != o->d || p->topk != o->topk ||
      p->score_dtype != (int)o->score_dtype || p->seed != o->seed || p->sigma != o->sigma ||
      p->solve.max_iter != o->solve.max_iter || p->solve.rel_tol != o->solve.rel_tol ||
      p->solve.flags != o->solve.flags)
    return false;
  return std::equal(p->n.begin(), p->n.end(), n);
}

template <typename T>
int upload(cudaStream_t s, T* dst, const std::vector<T>& v) {
  if (v.empty()) return CDL_OK;
  CDL_CUDA_TRY(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return CDL_OK;
}

int build_plan(cdl_ctx* ctx, int G, const int64_t* n, int T, const cdl_batch_opts* o, BatchPlan** out) {
  BatchPlan* P = new BatchPlan();
  P->G = G;
  P->T = T;
  P->k = o->k;
  P->d = o->d;
  P->topk = o->topk;
  P->score_dtype = (int)o->score_dtype;
  P->n.assign(n, n + G);
  P->seed = o->seed;
  P->sigma = o->sigma;
  P->solve = o->solve;
  const int G2 = 2 * G, k = o->k, d = o->d;
  const int kp = (int)round_up(k, 16);
  P->off.resize(G);
  for (int p = 0; p < G; ++p) {
    P->off[p] = P->N;
    P->N += n[p];
  }
  auto gn = [&](int g) { return (int)n[g / 2]; };
  auto gnp = [&](int g) { return (int)round_up(gn(g), 128); };
  P->order.resize(G2);
  std::iota(P->order.begin(), P->order.end(), 0);
  std::stable_sort(P->order.begin(), P->order.end(), [&](int a, int b) { return gn(a) > gn(b); });

  // ---- memory: two passes over the same carving sequence
  std::vector<BGraph> gs(G2);
  std::vector<ScoreJob> jobs(G);
  std::vector<double*> ab(G);
  std::vector<double*> contrib(G);
  P->chains.assign(G2, cdl_chain());
  P->A.assign(G2, nullptr);
  P->Dv.assign(G2, nullptr);
  P->scal.assign(G2, nullptr);
  P->Y.assign(G2, nullptr);
  const int n_sq_groups = std::max(d - 1, 1) * G2;
  const int n_lvl_groups = d * G2;
  TcGroup *lvl_groups = nullptr, *res_groups = nullptr;
  BGraph* d_gs = nullptr;
  BState* d_st = nullptr;
  uint32_t* d_tiles = nullptr;
  // tile tables (host)
  std::vector<uint32_t> t32, elem, csb, sel, spairs, snodes;
  std::vector<int> npads(G2), ns(G2);
  for (int g = 0; g < G2; ++g) {
    npads[g] = gnp(g);
    ns[g] = gn(g);
  }
  // squaring variants: 128 x 128 tiles up to a graph order (always where the
  // padded order is not a multiple of 256), 128 x 256 tiles above it
  const int thresholds[4] = {0, 1024, 2048, 32768};
  std::vector<std::vector<int>> sq_bn;
  for (int th : thresholds) {
    std::vector<int> bn(G2);
    for (int g = 0; g < G2; ++g) bn[g] = (npads[g] % 256 || npads[g] <= th) ? 128 : 256;
    if (!sq_bn.empty() && sq_bn.back() == bn) continue;
    sq_bn.push_back(bn);
    BatchPlan::SqVariant v;
    v.max_npad_128 = th;
    P->sqv.push_back(v);
  }
  std::vector<std::vector<uint32_t>> sq;
  for (auto& bn : sq_bn) sq.push_back(tc_grouped_square_tiles(npads, ns, bn));
  if (pair_clusters(ctx) > 0) {   // and every graph on CTA pairs
    sq_bn.push_back(std::vector<int>(G2, 128));
    sq.push_back(pair_tiles_grouped(npads, ns));
    BatchPlan::SqVariant v;
    v.max_npad_128 = -1;
    P->sqv.push_back(v);
  }
  const std::vector<uint32_t> ap = tc_grouped_apply_tiles(npads);
  const int kg = (int)round_up(k, 32);   // Z slice rows of the exact residual
  std::vector<uint32_t> cvec, cinit, zst, runits;
  for (int g : P->order) {
    const int nn = gn(g), np = gnp(g);
    for (int b = 0; b < (np + 255) / 256; ++b) cvec.push_back(((uint32_t)b << 12) | (uint32_t)g);
    for (size_t b = 0; b * 2048 < (size_t)np * (np / 8); ++b) cinit.push_back(((uint32_t)b << 12) | (uint32_t)g);
    for (int b = 0; b < np / 32; ++b) t32.push_back(((uint32_t)b << 12) | (uint32_t)g);
    const int eb = (int)(((size_t)nn * k + 255) / 256);
    for (int b = 0; b < eb; ++b) elem.push_back(((uint32_t)b << 12) | (uint32_t)g);
    for (size_t b = 0; b * 256 < (size_t)kg * np; ++b) zst.push_back(((uint32_t)b << 12) | (uint32_t)g);
    for (int t = 0; t < np / 128; ++t) runits.push_back((uint32_t)g | ((uint32_t)t << 16));
    for (int b = 0; b < (nn + 255) / 256; ++b) csb.push_back(((uint32_t)b << 12) | (uint32_t)g);
  }
  std::vector<int> porder(G);
  std::iota(porder.begin(), porder.end(), 0);
  std::stable_sort(porder.begin(), porder.end(), [&](int a, int b) { return n[a] > n[b]; });
  for (int p : porder) {
    const int nn = (int)n[p], nb = (nn + 63) / 64;
    const int eb = (int)(((size_t)nn * k + 255) / 256);
    for (int b = 0; b < eb; ++b) sel.push_back(((uint32_t)b << 12) | (uint32_t)p);
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj) spairs.push_back((uint32_t)p | ((uint32_t)bi << 12) | ((uint32_t)bj << 22));
    for (int b = 0; b < (nn + 255) / 256; ++b) snodes.push_back(((uint32_t)b << 12) | (uint32_t)p);
  }
  GraphTiles gt;
  {
    std::vector<int> gns(G2);
    for (int g = 0; g < G2; ++g) gns[g] = gn(g);
    graph_grouped_tiles(gns, T, gt);
  }
  // projection variants: node rows per block
  std::vector<std::vector<uint32_t>> pblocks;
  for (int rpb = project_rows_per_block(k); rpb >= 16; rpb /= 2) {
    std::vector<uint32_t> v;
    for (int g : P->order)
      for (int b = 0; b * rpb < gn(g); ++b) v.push_back(((uint32_t)b << 12) | (uint32_t)g);
    pblocks.push_back(std::move(v));
    BatchPlan::ProjVariant pvar;
    pvar.rpb = rpb;
    P->pv.push_back(pvar);
  }
  size_t ntiles = ap.size() + t32.size() + elem.size() + zst.size() + runits.size() + csb.size() + sel.size() +
                  spairs.size() + snodes.size() + gt.fixed.size() + gt.dist.size() + gt.rows.size() + cvec.size() +
                  cinit.size();
  for (auto& v : sq) ntiles += v.size();
  for (auto& v : pblocks) ntiles += v.size();
  std::vector<GGraph> ggs(G2);
  std::vector<PGraph> pgs(G2);
  std::vector<CGraph> cgs(G2);
  GGraph* d_ggs = nullptr;
  PGraph* d_pgs = nullptr;
  CGraph* d_cgs = nullptr;
  int4* d_sel = nullptr;
  char* sel_all = nullptr;
  ResidGroup* d_rgroups = nullptr;
  unsigned long long* zmax_all = nullptr;
  const size_t sel_one = graph_select_bytes();

  for (int pass = 0; pass < 2; ++pass) {
    Carver c;
    c.base = pass ? static_cast<char*>(P->mem) : nullptr;
    P->X = c.take<double>((size_t)2 * P->N * T);
    P->F = c.take<double>((size_t)P->N);
    P->top = c.take<int64_t>((size_t)G * std::max(o->topk, 1));
    d_gs = c.take<BGraph>(G2);
    d_st = c.take<BState>(G2);
    P->jobs = c.take<ScoreJob>(G);
    P->cmax = c.take<unsigned>((size_t)G * 2 * k);
    P->active = c.take<int>(1);
    for (auto& v : P->sqv) v.groups = c.take<TcGroup>(n_sq_groups);
    lvl_groups = c.take<TcGroup>(n_lvl_groups);
    res_groups = c.take<TcGroup>(2 * G2);
    d_tiles = c.take<uint32_t>(ntiles);
    d_ggs = c.take<GGraph>(G2);
    d_pgs = c.take<PGraph>(G2);
    d_cgs = c.take<CGraph>(G2);
    d_sel = c.take<int4>(gt.sel.size());
    sel_all = c.take<char>(G2 * sel_one);
    d_rgroups = c.take<ResidGroup>(G2);
    zmax_all = c.take<unsigned long long>((size_t)G2 * k);
    for (int g = 0; g < G2; ++g) {
      const int nn = gn(g), np = gnp(g);
      const size_t nk = (size_t)nn * k;
      BGraph& B = gs[g];
      cdl_chain& ch = P->chains[g];
      ggs[g].Xt = c.take<int>((size_t)nn * T);
      P->A[g] = c.take<double>((size_t)nn * nn);
      P->Dv[g] = c.take<double>(np);
      P->scal[g] = c.take<double>(2);   // vol, sigma
      P->Y[g] = c.take<double>(nk);
      ch.levels = c.take<uint16_t>((size_t)d * np * np);
      ch.aop = c.take<uint16_t>((size_t)2 * np * np);
      cgs[g].aslices = c.take<uint16_t>((size_t)6 * np * np);
      ch.rsqrt_d = c.take<double>(np);
      cgs[g].u = c.take<double>(np);
      cgs[g].rsf = c.take<float>(np);
      cgs[g].uf = c.take<float>(np);
      B.Z = c.take<double>(nk);
      B.R = c.take<double>(nk);
      B.x = c.take<float>((size_t)np * kp);
      B.xop = c.take<uint16_t>((size_t)2 * kp * np);
      B.part = c.take<float>((size_t)np * 2 * kp);
      B.part2 = c.take<float>((size_t)np * 2 * kp);
      B.dz = c.take<float>((size_t)np * kp);
      B.dzop = c.take<uint16_t>((size_t)2 * kp * np);
      B.kg = kg;
      B.zmax = zmax_all ? zmax_all + (size_t)g * k : nullptr;
      B.zc = c.take<double>(k);
      B.zs = c.take<uint16_t>((size_t)6 * kg * np);
      B.Gp = c.take<double>((size_t)RESID_PAIRS * np * kg);
      B.elem_blocks = (int)((nk + 255) / 256);
      B.res_tiles = B.elem_blocks;   // the full residual leaves one partial sum per element block
      B.red = c.take<double>(B.elem_blocks);
      B.cs = c.take<double>((size_t)((nn + 255) / 256) * k);
    }
    for (int p = 0; p < G; ++p) {
      const int nn = (int)n[p];
      ab[p] = c.take<double>((size_t)2 * nn * k);   // 16 n k bytes
      contrib[p] = c.take<double>((size_t)((nn + 63) / 64) * nn);
    }
    if (pass == 0) {
      P->bytes = c.used;
      if (ctx->ws_cap && ctx->ws_used + P->bytes > ctx->ws_cap) {
        delete P;
        return CDL_ERR_OOM;
      }
      if (cudaMalloc(&P->mem, P->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return CDL_ERR_OOM;
      }
    }
  }
  // ---- private context and stream
  int st = CDL_OK;
  auto fail = [&](int s) {
    batch_plan_free(P);
    return s;
  };
  if (cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(CDL_ERR_CUDA);
  }
  st = cdl_ctx_create(&P->inner, ctx->device, P->stream, 0);
  if (st != CDL_OK) return fail(st);
  if (cudaMemsetAsync(P->mem, 0, P->bytes, P->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(CDL_ERR_CUDA);
  }
  // ---- per-graph descriptors, chains, tensor maps
  for (int g = 0; g < G2; ++g) {
    const int nn = gn(g), np = gnp(g);
    cdl_chain& ch = P->chains[g];
    ch.device = ctx->device;
    ch.n = nn;
    ch.npad = np;
    ch.d = d;
    ch.dtype = CDL_BF16;
    ch.elem = 2;
    ch.D = P->Dv[g];
    ch.vol = P->scal[g];
    BGraph& B = gs[g];
    B.n = nn;
    B.np = np;
    B.D = ch.D;
    B.rsd = ch.rsqrt_d;
    B.vol = ch.vol;
    B.Y = P->Y[g];
    GGraph& Gg = ggs[g];
    const int p = g / 2;
    Gg.X = P->X + ((g & 1) ? P->N : 0) * (size_t)T + P->off[p] * (size_t)T;
    Gg.A = P->A[g];
    Gg.D = P->Dv[g];
    Gg.vol = P->scal[g];
    Gg.sigma = P->scal[g] + 1;
    Gg.sel = sel_all + (size_t)g * sel_one;
    Gg.n = nn;
    Gg.T = T;
    CGraph& Cg = cgs[g];
    Cg.A = P->A[g];
    Cg.D = ch.D;
    Cg.vol = ch.vol;
    Cg.rsd = ch.rsqrt_d;
    Cg.L0 = ch.level(0);
    Cg.aop = ch.aop;
    Cg.n = nn;
    Cg.npad = np;
    P->cinit_bytes += 8.0 * nn * (double)nn + 18.0 * np * (double)np;   // A read; level 0, A hi/lo, 6 slices
    PGraph& Pg = pgs[g];
    Pg.A = P->A[g];
    Pg.Y = P->Y[g];
    Pg.part = B.cs;
    Pg.n = nn;
    Pg.pad = 0;
  }
  P->lvl_first.resize(d);
  P->res_first.resize(2);
  {
    std::vector<std::vector<TcGroup>> sqg(P->sqv.size(), std::vector<TcGroup>(n_sq_groups));
    std::vector<TcGroup> lvg(n_lvl_groups), rsg(2 * G2);
    std::vector<ResidGroup> rg(G2);
    for (int g = 0; g < G2; ++g) {
      const cdl_chain& ch = P->chains[g];
      const int np = (int)ch.npad;
      const int* gate = &d_st[g].cmd;
      for (size_t v = 0; v < P->sqv.size(); ++v)
        for (int l = 0; l + 1 < d; ++l)
          if ((st = tc_group_square(&sqg[v][(size_t)l * G2 + g], ch.level(l), ch.level(l + 1), np, sq_bn[v][g],
                                    gn(g))) != CDL_OK)
            return fail(st);
      for (int l = 0; l < d; ++l)
        if ((st = tc_group_apply(&lvg[(size_t)l * G2 + g], ch.level(l), gs[g].xop, gs[g].part, np, kp, gate)) !=
            CDL_OK)
          return fail(st);
      if ((st = resid_group_init(&rg[g], cgs[g].aslices, gs[g].zs, const_cast<double*>(gs[g].Gp), np, kg, gate)) !=
          CDL_OK)
        return fail(st);
      const uint16_t* aop = static_cast<const uint16_t*>(ch.aop);
      if ((st = tc_group_apply(&rsg[g], aop, gs[g].dzop, gs[g].part, np, kp, gate)) != CDL_OK ||
          (st = tc_group_apply(&rsg[G2 + g], aop + (size_t)np * np, gs[g].dzop, gs[g].part2, np, kp, gate)) !=
              CDL_OK)
        return fail(st);
    }
    for (size_t v = 0; v < P->sqv.size(); ++v) {
      P->sqv[v].first.resize(std::max(d - 1, 1));
      for (int l = 0; l + 1 < d; ++l) P->sqv[v].first[l] = sqg[v][(size_t)l * G2];
      if ((st = upload(P->stream, P->sqv[v].groups, sqg[v])) != CDL_OK) return fail(st);
    }
    for (int l = 0; l < d; ++l) P->lvl_first[l] = lvg[(size_t)l * G2];
    P->res_first[0] = rsg[0];
    P->res_first[1] = rsg[G2];
    if ((st = upload(P->stream, lvl_groups, lvg)) != CDL_OK ||
        (st = upload(P->stream, res_groups, rsg)) != CDL_OK || (st = upload(P->stream, d_rgroups, rg)) != CDL_OK)
      return fail(st);
    // the host vectors are read by the copies above: finish them before they go
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return fail(CDL_ERR_CUDA);
  }
  for (int p = 0; p < G; ++p) {
    ScoreJob& J = jobs[p];
    J.A1 = P->A[2 * p];
    J.A2 = P->A[2 * p + 1];
    J.Z1 = gs[2 * p].Z;
    J.Z2 = gs[2 * p + 1].Z;
    J.vol1 = P->scal[2 * p];
    J.vol2 = P->scal[2 * p + 1];
    J.ab = ab[p];
    J.contrib = contrib[p];
    J.F = P->F + P->off[p];
    J.top = P->top + (size_t)p * std::max(o->topk, 1);
    J.cmax = P->cmax + (size_t)p * 2 * k;
    J.n = (int)n[p];
    J.pad = 0;
  }
  // tile tables, in the carving order above
  std::vector<uint32_t> all;
  all.reserve(ntiles);
  auto add = [&](const std::vector<uint32_t>& v, BTiles& t) {
    t.p = d_tiles + all.size();
    t.count = (int)v.size();
    all.insert(all.end(), v.begin(), v.end());
  };
  BatchSolve& bs = P->bs;
  for (size_t v = 0; v < sq.size(); ++v) add(sq[v], P->sqv[v].tiles);
  add(ap, bs.apply);
  add(t32, bs.t32);
  add(elem, bs.elem);
  add(zst, bs.zst);
  add(runits, bs.runits);
  add(csb, bs.cs);
  add(sel, P->score_elem);
  add(spairs, P->score_pairs);
  add(snodes, P->score_nodes);
  GraphBatch& gb = P->gb;
  add(gt.fixed, gb.fixed);
  add(gt.dist, gb.dist);
  add(gt.rows, gb.rows);
  for (size_t v = 0; v < pblocks.size(); ++v) add(pblocks[v], P->pv[v].blocks);
  add(cvec, P->cvec);
  add(cinit, P->cinit);
  // before tuning: 128 x 128 tiles up to order 1024, the widest projection blocks
  P->sq_choice = std::min<int>(1, (int)P->sqv.size() - 1);
  P->pv_choice = 0;
  if ((st = upload(P->stream, d_tiles, all)) != CDL_OK || (st = upload(P->stream, d_gs, gs)) != CDL_OK ||
      (st = upload(P->stream, P->jobs, jobs)) != CDL_OK || (st = upload(P->stream, d_ggs, ggs)) != CDL_OK ||
      (st = upload(P->stream, d_pgs, pgs)) != CDL_OK || (st = upload(P->stream, d_sel, gt.sel)) != CDL_OK ||
      (st = upload(P->stream, d_cgs, cgs)) != CDL_OK)
    return fail(st);
  P->cgs = d_cgs;
  gb.G2 = G2;
  gb.sigma = o->sigma;
  gb.gs = d_ggs;
  gb.sel_all = sel_all;
  gb.sel_bytes = (size_t)G2 * sel_one;
  gb.sel = d_sel;
  gb.sel_count = (int)gt.sel.size();
  P->pgs = d_pgs;
  for (int g = 0; g < G2; ++g) {
    const double nn = gn(g);
    gb.dist_terms += 0.5 * nn * (nn - 1) * T;
    gb.select_bytes += 8.0 * nn * (nn - 1) / 2;
    gb.kernel_bytes += 16.0 * nn * nn;
    P->proj_adds += nn * (nn - 1) * k;
  }
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return fail(CDL_ERR_CUDA);
  bs.G2 = G2;
  bs.k = k;
  bs.kp = kp;
  bs.d = d;
  bs.max_iter = o->solve.max_iter;
  bs.rel_tol = o->solve.rel_tol;
  bs.always_full = (o->solve.flags & CDL_SOLVE_FULL_RESIDUAL) != 0;
  // one slot is one refinement step or one certification of a recursively
  // updated residual; four slots beyond max_iter leave room for those
  bs.max_slots = o->solve.max_iter + (bs.always_full ? 0 : 4);
  bs.gs = d_gs;
  bs.st = d_st;
  bs.active = P->active;
  bs.lvl_groups = lvl_groups;
  bs.lvl_first = P->lvl_first.data();
  bs.res_groups = res_groups;
  bs.res_first = P->res_first.data();
  bs.rgroups = d_rgroups;
  bs.zmax_all = zmax_all;
  bs.zmax_bytes = (size_t)G2 * k * sizeof(unsigned long long);
  bs.kg = kg;
  for (int g = 0; g < G2; ++g) {
    const double np = gnp(g);
    bs.apply_bytes += 2.0 * np * np;
    bs.resid_work += 2.0 * RESID_PAIRS * np * np * kg;
    P->sq_flops += (double)gn(g) * gn(g) * (gn(g) + 1.0);
  }
  for (int p = 0; p < G; ++p) P->score_bytes += 8.0 * (double)n[p] * (n[p] - 1);
  P->st_host.resize(G2);
  *out = P;
  return CDL_OK;
}

// Refinement slots run eagerly until no graph is still refining (the count of
// running graphs is read back after each slot) or the slot budget is spent.
int solve_adaptive(BatchPlan* P, int done, int* used) {
  cdl_ctx* c = P->inner;
  int s = done;
  while (s < P->bs.max_slots) {
    CDL_TRY(batch_solve_slot(c, P->bs));
    ++s;
    int running = 0;
    CDL_CUDA_TRY(cudaMemcpyAsync(&running, P->active, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    CDL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    if (running == 0) break;
  }
  *used = s;
  return CDL_OK;
}

int score_batch(BatchPlan* P) {
  return cad_score_grouped(P->inner, P->jobs, P->G, P->k, P->score_dtype == CDL_F64, P->topk, P->score_elem,
                           P->score_pairs, P->score_nodes, P->score_bytes, P->cmax);
}

// The whole batch on the plan's private context. fixed_slots > 0 issues that
// many refinement slots with no host synchronisation (the form recorded as a
// CUDA graph); 0 runs them adaptively.
// Level l -> l + 1 of every graph in one launch of a squaring variant.
int square_variant(cdl_ctx* c, const BatchPlan::SqVariant& sv, int l, int G2, double flops) {
  if (sv.max_npad_128 < 0)
    return tc_square_grouped_pairs(c, &sv.first[l], sv.groups + (size_t)l * G2, sv.tiles.p, sv.tiles.count, flops);
  return tc_square_grouped(c, &sv.first[l], sv.groups + (size_t)l * G2, sv.tiles.p, sv.tiles.count, flops);
}

int run_batch(BatchPlan* P, int fixed_slots) {
  cdl_ctx* c = P->inner;
  const int G2 = 2 * P->G;
  CDL_TRY(graph_build_grouped(c, P->gb));
  CDL_TRY(chain_init_grouped(c, P->cgs, P->cvec, P->cinit, P->cinit_bytes));
  const BatchPlan::SqVariant& sv = P->sqv[P->sq_choice];
  for (int l = 0; l + 1 < P->d; ++l)
    CDL_TRY(square_variant(c, sv, l, G2, P->sq_flops));
  const BatchPlan::ProjVariant& pvar = P->pv[P->pv_choice];
  CDL_TRY(project_grouped(c, P->pgs, G2, pvar.blocks, pvar.rpb, P->k, P->seed, P->bs.cs, P->bs.elem,
                          P->proj_adds));
  CDL_TRY(batch_solve_start(c, P->bs));
  if (fixed_slots > 0) {
    for (int s = 0; s < fixed_slots; ++s) CDL_TRY(batch_solve_slot(c, P->bs));
  } else {
    int used = 0;
    CDL_TRY(solve_adaptive(P, 0, &used));
    P->slots_seen = std::max(P->slots_seen, used);
  }
  return score_batch(P);
}

// Autotuner: times each squaring variant (level 0 -> 1 of every graph) and
// each projection variant on the batch's own data, after a first run has
// filled the buffers, and keeps the fastest. The kernels it reruns are pure
// functions of buffers the rerun does not change (level 0, A), and the
// buffers they write are formed again by every later run.
int autotune(BatchPlan* P) {
  cdl_ctx* c = P->inner;
  const bool timing = c->timing;
  c->timing = false;
  cudaEvent_t e0, e1;
  CDL_CUDA_TRY(cudaEventCreate(&e0));
  CDL_CUDA_TRY(cudaEventCreate(&e1));
  auto time_it = [&](auto&& fn, double* ms) -> int {
    CDL_TRY(fn());   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      CDL_CUDA_TRY(cudaEventRecord(e0, P->stream));
      CDL_TRY(fn());
      CDL_CUDA_TRY(cudaEventRecord(e1, P->stream));
      CDL_CUDA_TRY(cudaEventSynchronize(e1));
      float t = 0.f;
      CDL_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
      best = std::min(best, t);
    }
    *ms = best;
    return CDL_OK;
  };
  const int G2 = 2 * P->G;
  int st = CDL_OK;
  if (P->d > 1)
    for (size_t v = 0; v < P->sqv.size() && st == CDL_OK; ++v) {
      BatchPlan::SqVariant& sv = P->sqv[v];
      st = time_it([&] { return square_variant(c, sv, 0, G2, 0.0); }, &sv.ms);
    }
  for (size_t v = 0; v < P->pv.size() && st == CDL_OK; ++v) {
    BatchPlan::ProjVariant& pvar = P->pv[v];
    st = time_it([&] { return project_grouped(c, P->pgs, G2, pvar.blocks, pvar.rpb, P->k, P->seed, P->bs.cs,
                                              P->bs.elem, 0.0); },
                 &pvar.ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = timing;
  // tuning launches are not part of any call's work
  c->launches = 0;
  for (int i = 0; i < CDL_KC_COUNT; ++i) c->kc_launches[i] = 0, c->kc_work[i] = 0, c->kc_ms[i] = 0;
  CDL_TRY(st);
  if (P->d > 1)
    for (size_t v = 0; v < P->sqv.size(); ++v)
      if (P->sqv[v].ms < P->sqv[P->sq_choice].ms) P->sq_choice = (int)v;
  for (size_t v = 0; v < P->pv.size(); ++v)
    if (P->pv[v].ms < P->pv[P->pv_choice].ms) P->pv_choice = (int)v;
  P->tuned = true;
  return CDL_OK;
}

int capture(BatchPlan* P, int slots) {
  cdl_ctx* c = P->inner;
  const bool timing = c->timing;
  c->timing = false;
  const int64_t l0 = c->launches;
  int64_t kl0[CDL_KC_COUNT];
  double kw0[CDL_KC_COUNT];
  for (int i = 0; i < CDL_KC_COUNT; ++i) {
    kl0[i] = c->kc_launches[i];
    kw0[i] = c->kc_work[i];
  }
  CDL_CUDA_TRY(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
  const int st = run_batch(P, slots);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(P->stream, &graph);
  c->timing = timing;
  P->graph_launches = c->launches - l0;
  c->launches = l0;
  for (int i = 0; i < CDL_KC_COUNT; ++i) {
    P->graph_kc_launches[i] = c->kc_launches[i] - kl0[i];
    P->graph_kc_work[i] = c->kc_work[i] - kw0[i];
    c->kc_launches[i] = kl0[i];
    c->kc_work[i] = kw0[i];
  }
  if (st != CDL_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (e != cudaSuccess) set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return st != CDL_OK ? st : CDL_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&P->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    P->exec = nullptr;
    cudaGetLastError();
    set_last_error(cudaGetErrorString(ei), __FILE__, __LINE__);
    return CDL_ERR_CUDA;
  }
  P->slots_captured = slots;
  return CDL_OK;
}

}  // namespace
}  // namespace cdl

using namespace cdl;

extern "C" int cdl_caddelag_batched(cdl_ctx* ctx, int32_t G, const int64_t* n, int32_t T, const double* X1,
                                    const double* X2, const cdl_batch_opts* o, double* F, int64_t* top_idx,
                                    cdl_solve_stats* stats) {
  if (!ctx || !n || !o || !X1 || !X2 || !F) return CDL_ERR_INVALID_ARG;
  if (G < 1 || G > 2048 || T < 1 || T > 4096 || o->k < 1 || o->k > 128 || o->d < 1 || o->d > 64 ||
      o->chain_dtype != CDL_BF16 || (o->score_dtype != CDL_F64 && o->score_dtype != CDL_F32) || o->topk < 0 ||
      o->topk > 1024 || (o->topk > 0 && !top_idx) || o->solve.max_iter < 1 || o->solve.max_iter > 1000 ||
      o->solve.rel_tol < 0 || (o->solve.flags & ~CDL_SOLVE_FULL_RESIDUAL) != 0)
    return CDL_ERR_INVALID_ARG;
  int64_t N = 0;
  for (int p = 0; p < G; ++p) {
    if (n[p] < 2 || n[p] > 32768 || o->topk > n[p]) return CDL_ERR_INVALID_ARG;
    N += n[p];
  }
  if (N > (int64_t)1 << 26) return CDL_ERR_INVALID_ARG;
  CDL_CUDA_TRY(cudaSetDevice(ctx->device));
  if (!o->host_io) {
    CDL_TRY(check_dev_ptr(ctx, X1, 8));
    CDL_TRY(check_dev_ptr(ctx, X2, 8));
    CDL_TRY(check_dev_ptr(ctx, F, 8));
    if (o->topk > 0) CDL_TRY(check_dev_ptr(ctx, top_idx, 8));
  }
  if (!tc_supported(ctx)) return CDL_ERR_UNSUPPORTED;
  if (!same_key(ctx->batch, G, n, T, o)) {
    if (ctx->batch) {
      CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      batch_plan_free(ctx->batch);
      ctx->batch = nullptr;
    }
    CDL_TRY(build_plan(ctx, G, n, T, o, &ctx->batch));
    if (ctx->debug_flags & CDL_DEBUG_BATCH_VARIANT) {
      BatchPlan* Q = ctx->batch;
      Q->sq_choice = std::min((ctx->debug_flags >> 8) & 15, (int)Q->sqv.size() - 1);
      Q->pv_choice = std::min((ctx->debug_flags >> 12) & 15, (int)Q->pv.size() - 1);
      Q->tuned = true;
    }
  }
  BatchPlan* P = ctx->batch;
  cudaStream_t s = P->stream;
  const cudaMemcpyKind in = o->host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind outk = o->host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CDL_CUDA_TRY(cudaEventRecord(P->ev_in, ctx->stream));
  CDL_CUDA_TRY(cudaStreamWaitEvent(s, P->ev_in, 0));
  const size_t xbytes = (size_t)N * T * sizeof(double);
  CDL_CUDA_TRY(cudaMemcpyAsync(P->X, X1, xbytes, in, s));
  CDL_CUDA_TRY(cudaMemcpyAsync(P->X + (size_t)N * T, X2, xbytes, in, s));
  P->inner->timing = ctx->timing;
  P->inner->debug_flags = 0;
  bool replayed = false;
  const bool graph_current =
      P->exec && (P->slots_captured > P->slots_seen || P->slots_captured >= P->bs.max_slots);
  if (o->use_graph && graph_current) {
    CDL_CUDA_TRY(cudaGraphLaunch(P->exec, s));
    replayed = true;
    ctx->launches += P->graph_launches;
    for (int i = 0; i < CDL_KC_COUNT; ++i) {
      ctx->kc_launches[i] += P->graph_kc_launches[i];
      ctx->kc_work[i] += P->graph_kc_work[i];
    }
  } else {
    CDL_TRY(run_batch(P, 0));
    if (!P->tuned) {
      // count this run's launches before the tuner's reruns
      CDL_CUDA_TRY(cudaStreamSynchronize(s));
      CDL_TRY(ctx_absorb(ctx, P->inner));
      CDL_TRY(autotune(P));
    }
    if (o->use_graph) {
      if (P->exec) {
        CDL_CUDA_TRY(cudaGraphExecDestroy(P->exec));
        P->exec = nullptr;
      }
      // one slot beyond the most any call has needed
      CDL_TRY(capture(P, std::min(P->slots_seen + 1, P->bs.max_slots)));
    }
  }
  if (replayed) {
    // graphs still refining after the recorded slots continue eagerly (and
    // the graph is recorded again with more slots on the next call)
    int running = 0;
    CDL_CUDA_TRY(cudaMemcpyAsync(&running, P->active, sizeof(int), cudaMemcpyDeviceToHost, s));
    CDL_CUDA_TRY(cudaStreamSynchronize(s));
    if (running > 0 && P->slots_captured < P->bs.max_slots) {
      int used = 0;
      CDL_TRY(solve_adaptive(P, P->slots_captured, &used));
      P->slots_seen = std::max(P->slots_seen, used);
      CDL_TRY(score_batch(P));
    }
  }
  CDL_CUDA_TRY(cudaMemcpyAsync(F, P->F, (size_t)N * sizeof(double), outk, s));
  if (o->topk > 0)
    CDL_CUDA_TRY(cudaMemcpyAsync(top_idx, P->top, (size_t)G * o->topk * sizeof(int64_t), outk, s));
  CDL_CUDA_TRY(cudaMemcpyAsync(P->st_host.data(), P->bs.st, P->st_host.size() * sizeof(BState),
                               cudaMemcpyDeviceToHost, s));
  unsigned dev_status = 0;
  CDL_CUDA_TRY(cudaMemcpyAsync(&dev_status, P->inner->dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CDL_CUDA_TRY(cudaStreamSynchronize(s));
  CDL_TRY(ctx_absorb(ctx, P->inner));
  if (dev_status != DEV_OK) {
    CDL_CUDA_TRY(cudaMemset(P->inner->dev_status, 0, sizeof(unsigned)));
    return CDL_ERR_TIMEOUT;
  }
  bool converged = true;
  for (int g = 0; g < 2 * G; ++g) {
    const BState& b = P->st_host[g];
    const bool ok = b.cmd == 0 && (b.rel <= 1e6) && !(o->solve.rel_tol > 0 && !(b.rel <= o->solve.rel_tol));
    converged = converged && ok;
    if (stats) {
      stats[g].iters = b.iters;
      stats[g].rel_res = b.rel;
      for (int h = 0; h < 64; ++h) stats[g].history[h] = b.hist[h];
    }
  }
  return converged ? CDL_OK : CDL_ERR_NOT_CONVERGED;
}

extern "C" int cdl_batch_plan_info(const cdl_ctx* ctx, cdl_batch_info* info) {
  if (!ctx || !info) return CDL_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  const BatchPlan* P = ctx->batch;
  if (!P) return CDL_OK;
  info->ready = 1;
  info->square_max_npad_128 = P->sqv[P->sq_choice].max_npad_128;
  info->project_rows_per_block = P->pv[P->pv_choice].rpb;
  int tm, tn;
  batch_residual_tile(P->k, &tm, &tn);
  info->residual_tile_m = tm;
  info->residual_tile_n = tn;
  info->slots_captured = P->exec ? P->slots_captured : 0;
  info->slots_seen = P->slots_seen;
  info->n_square_variants = (int)std::min<size_t>(8, P->sqv.size());
  info->n_project_variants = (int)std::min<size_t>(8, P->pv.size());
  for (int v = 0; v < info->n_square_variants; ++v) {
    info->square_variant_max_npad_128[v] = P->sqv[v].max_npad_128;
    info->square_variant_ms[v] = P->sqv[v].ms;
  }
  for (int v = 0; v < info->n_project_variants; ++v) {
    info->project_variant_rows[v] = P->pv[v].rpb;
    info->project_variant_ms[v] = P->pv[v].ms;
  }
  info->device_bytes = P->bytes;
  return CDL_OK;
}
