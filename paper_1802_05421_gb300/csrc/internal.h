// Library-internal declarations shared by the translation units of libcdl.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <functional>
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

namespace cdl {
struct BatchPlan;
void batch_plan_free(BatchPlan* p);
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
  cdl_chain* regen_chain = nullptr;   // the chain of pairs whose graphs are regenerated in panels
  // where the last cdl_caddelag_pair left its embeddings (workspace, device)
  struct {
    int64_t n = 0;
    int k = 0;
    const double* Z[2] = {nullptr, nullptr};
    const double* vol[2] = {nullptr, nullptr};
    const double* sigma[2] = {nullptr, nullptr};
  } last_pair;
  // tile schedules uploaded to the workspace, by workspace name -> tile count
  std::map<std::string, int> tile_lists;
  int debug_flags = 0;   // CDL_DEBUG_* test hooks
  cdl::BatchPlan* batch = nullptr;   // plan of the last cdl_caddelag_batched call
  // one-shot hint from the pair driver: the device float64 bits of max |A| of the
  // graph at amax_hint_A (found while its kernel values were formed), taken and
  // cleared by the next chain build of that graph instead of a pass over A
  const double* amax_hint_A = nullptr;
  const unsigned long long* amax_hint_bits = nullptr;
};

namespace cdl {
struct RegenSource;
}

struct cdl_chain {
  int device = 0;
  int64_t n = 0, npad = 0;
  int32_t d = 0;
  int32_t d_eff = 0;          // levels in use (d unless CDL_CHAIN_TRUNCATE stopped earlier)
  cdl_dtype dtype = CDL_F64;
  size_t elem = 8;
  void* levels = nullptr;     // d * npad * npad elements
  void* aop = nullptr;        // bf16 chains: A = A_hi + A_lo as two bf16 npad x npad matrices
  void* levels16 = nullptr;   // fp8 chains: bf16 copies of the levels (the apply's operand)
  unsigned* amax = nullptr;   // fp8 chains: per-level bound of |value| (float bits), scale = amax/448
  float* ahl = nullptr;       // A as float hi + lo planes (n x n each), the float-float residual's operand
  float* tscale = nullptr;    // per-tile e4m3 chains: d x (npad/128)^2 tile scales (powers of two)
  uint8_t* tatoms = nullptr;  // per-tile e4m3 chains: two (ping-pong by level parity) sets of
                              // (npad/128)^2 512-byte atoms, each the tile's e8m0 scale byte repeated
  void* aslices = nullptr;    // tensor chains: A / a_scale as 6 bf16 planes npad x npad on the grids 2^-8s
  double* a_scale = nullptr;  // tensor chains (device, 2 words): [0] the power of two >= max A that the
                              // slices are taken of, [1] the float64 bits of max |A|
  double* rsqrt_d = nullptr;  // npad: D_i^{-1/2} (0 in padding)
  double* D = nullptr;        // npad: degrees (0 in padding)
  double* vol = nullptr;      // 1
  // CDL_CHAIN_HOST_LEVELS: levels 0 .. resident - 1 in device memory
  // (dev_levels), the others in pinned host memory (`levels`, level i at
  // (i - resident) npad^2); two device slots hold the host levels in use,
  // filled and drained on a copy stream.
  bool host_levels = false;
  int resident = 0;
  void* dev_levels = nullptr;
  void* slot[2] = {nullptr, nullptr};
  int slot_level[2] = {-1, -1};
  int last_level = -1;                            // level written or read last
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_ready[2] = {nullptr, nullptr};   // slot content complete
  cudaEvent_t ev_free[2] = {nullptr, nullptr};    // slot's last copy-out or reader done
  double link_bytes = 0;                          // host <-> device bytes moved
  // Graphs not kept (cdl_caddelag_pair with CDL_PAIR_REGEN_GRAPHS): the solve
  // forms A Z from the graph regenerated panel by panel.
  const cdl::RegenSource* regen = nullptr;
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

// *out (device) = the float64 bit pattern of max |x_i| over count values
// (asynchronous; out is zeroed first).
int abs_max_bits(cdl_ctx* ctx, const double* x, size_t count, unsigned long long* out);

// Folds src's pending timings and adds its launch counters into dst, then
// zeroes src's counters.
int ctx_absorb(cdl_ctx* dst, cdl_ctx* src);
// CDL_OK if p is device (or managed) memory of ctx's device, aligned to `align`.
int check_dev_ptr(const cdl_ctx* ctx, const void* p, size_t align);

// Launch accounting: call before and after each kernel launch.
struct Launch {
  cdl_ctx* ctx;
  int kc;
  double work;
  cudaEvent_t a = nullptr;
  Launch(cdl_ctx* c, int k, double w);
  int done();   // checks cudaGetLastError, records the end event
};

// Timing of one host-link copy on stream `s` (class CDL_KC_HOST_LINK): events
// around it when timing is on; counted as a copy, not as a kernel launch.
struct CopyTimer {
  cdl_ctx* ctx;
  cudaStream_t s;
  double bytes;
  cudaEvent_t a = nullptr;
  CopyTimer(cdl_ctx* c, cudaStream_t st, double b);
  void done();
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---- kernel launchers (one per translation unit family) ----
// graph.cu
// amax_bits (device, optional): receives the float64 bits of max A.
int graph_build(cdl_ctx* ctx, const double* X, int64_t n, int T, double sigma, double* A,
                double* D, double* vol, double* sigma_out, int kernel = 0,
                unsigned long long* amax_bits = nullptr);
int graph_degrees(cdl_ctx* ctx, const double* A, int64_t n, double* D, double* vol);
int graph_add_edges(cdl_ctx* ctx, double* A, int64_t n, int64_t m, const int64_t* ij, const double* w,
                    int64_t* n_bad);
int graph_build_static(const double* X, int64_t n, int T, double sigma, double* A, double* D,
                       double* vol, double* sigma_out, cudaStream_t stream);
// chain.cu
int chain_init(cdl_ctx* ctx, cdl_chain* ch, const double* A);
int chain_square_simt(cdl_ctx* ctx, cdl_chain* ch, int level);
int fp8_level_bound(cdl_ctx* ctx, cdl_chain* ch, int level);
// Max absolute row sum of level i (an upper bound of its spectral norm, the
// level being symmetric), as float bits in *out_bits (device).
int level_inf_norm(cdl_ctx* ctx, const cdl_chain* ch, int level, unsigned* out_bits);
int apply_simt(cdl_ctx* ctx, const cdl_chain* ch, int level, const void* x, void* partial,
               int k, int splits);
// ooc.cu: levels in pinned host memory (bf16 chains), the first ch->resident
// of them in device memory
int ooc_init(cdl_chain* ch);
void ooc_destroy(cdl_chain* ch);
// Where level i lives (device pointer for resident levels, else host).
void* ooc_level_ptr(const cdl_chain* ch, int i);
// Device slot to write level i into (waits until the slot's old level is
// saved and read); ooc_write_end saves it to the host on the copy stream.
void* ooc_write_begin(cdl_ctx* ctx, cdl_chain* ch, int i);
int ooc_write_end(cdl_ctx* ctx, cdl_chain* ch, int i);
// Device copy of level i for reading on ctx->stream (loaded if no slot holds
// it); ooc_read_done marks the end of the reads; ooc_prefetch starts a load
// without waiting for it.
const void* ooc_read(cdl_ctx* ctx, cdl_chain* ch, int i);
int ooc_read_done(cdl_ctx* ctx, cdl_chain* ch, int i);
int ooc_prefetch(cdl_ctx* ctx, cdl_chain* ch, int i);
// tc_gemm.cu
int chain_square_tc(cdl_ctx* ctx, cdl_chain* ch, int level);
// Number of exact-slice pairs of the residual product (s + t <= 7 of six slices).
constexpr int RESID_PAIRS = 21;
// A Z on the tensor cores from exact bf16 slices (A's in the chain, Z / c in
// zslices: 6 planes kp x npad) into G: RESID_PAIRS float64 planes npad x kp,
// one per slice pair; A Z = the sum of the planes in order.
int resid_tc(cdl_ctx* ctx, const cdl_chain* ch, const void* zslices, int kp, double* G);
// The same product for many graphs in one launch (batched form): each graph's
// A slice planes (6 x npad x npad, npad a multiple of 128), Z slice planes
// (6 x kg x npad) and RESID_PAIRS output planes (npad x kg, assigned, not
// added: no zeroing needed) sit in a device array of ResidGroup; units lists
// graph | row tile << 16 for every 128-row tile of every graph; a graph's
// units run iff *gate & gate_mask.
struct ResidGroup {
  CUtensorMap a[6];    // A slice planes, 128-row boxes
  CUtensorMap b[6];    // Z slice planes (transposed, kg x npad), kg-row boxes
  double* G;
  size_t gstride;      // npad x kg
  const int* gate;
  int kblocks;         // npad rounded up to 256, in 64-wide k-blocks (zero fill past npad)
  int pad[9];
};
static_assert(sizeof(ResidGroup) % 64 == 0, "ResidGroup keeps its tensor maps 64-byte aligned in arrays");
int resid_group_init(ResidGroup* g, const void* aslices, const void* zslices, double* G, int npad, int kg,
                     const int* gate);
int resid_tc_grouped(cdl_ctx* ctx, const ResidGroup* dgroups, const uint32_t* units, int nunits, int kg,
                     int gate_mask, double work);
// Exact squared distances of grid inputs on the tensor cores: planes = three
// bf16 digit planes (rows x tp each, rows = n rounded up to 128, tp = T
// rounded up to 64, zero padded), norms = |a_i|^2 (rows, int64); writes the
// n x n float64 matrix A unless *offgrid & 1; terms = the algorithmic work
// recorded for the launch.
int dist_tc(cdl_ctx* ctx, const void* planes, const long long* norms, int n, int rows, int tp, double* A,
            const int* offgrid, double terms);
// Pair partials of the CAD scores with the Gram on the tensor cores: uplanes,
// vplanes = six bf16 slice planes each (rows x k2p, zero padded) of u / c and
// v / c; dint = d_i in units of c^2 2^-48; oscale = c^2 2^-48 (device);
// writes contrib (64-node partner blocks x n) for k_score_reduce.
int score_tc(cdl_ctx* ctx, const void* uplanes, const void* vplanes, const long long* dint, const double* oscale,
             int n, int rows, int k2p, const double* A1, const double* A2, double* contrib);
int chain_square_fp8t(cdl_ctx* ctx, cdl_chain* ch, int level);
int fp8t_quantize_level0(cdl_ctx* ctx, cdl_chain* ch);
// Grouped (batched) tcgen05 launches: one launch over the tiles of many
// graphs. Each graph's tensor maps, output and k-loop length sit in a device
// array of TcGroup; `host_first` is the host copy of entry 0.
struct TcGroup {
  CUtensorMap mapA;    // A operand (128-row boxes)
  CUtensorMap mapB;    // B operand
  void* out;           // squaring: bf16 level; apply: float npad x 2kp
  const int* gate;     // apply: tiles run iff *gate & gate_mask (null: always)
  int npad;
  int kblocks;
  uint32_t idesc;      // tcgen05 instruction descriptor of this graph's tiles
  int bn;              // MMA N: squaring 128 or 256, apply 2 kp
  int pad[8];
};
static_assert(sizeof(TcGroup) % 64 == 0, "TcGroup keeps its tensor maps 64-byte aligned in arrays");
// bn = 256: 128 x 256 tiles in 256-blocks (npad % 256 == 0); bn = 128:
// 128 x 128 tiles (npad % 128 == 0).
int tc_group_square(TcGroup* g, const void* level, void* out, int np, int bn, int n);
int tc_group_apply(TcGroup* g, const void* amat, const void* xop, float* out, int np, int kp, const int* gate);
std::vector<uint32_t> tc_grouped_square_tiles(const std::vector<int>& npad, const std::vector<int>& n,
                                              const std::vector<int>& bn);
std::vector<uint32_t> tc_grouped_apply_tiles(const std::vector<int>& npad);
int tc_square_grouped(cdl_ctx* ctx, const TcGroup* host_first, const TcGroup* dgroups, const uint32_t* dtiles,
                      int ntiles, double flops);
// The same squarings on CTA pairs (256 x 256 blocks, tcgen05.mma.cta_group::2);
// uses each group's mapA (128-row boxes), out, npad and kblocks.
std::vector<uint32_t> pair_tiles_grouped(const std::vector<int>& npad, const std::vector<int>& n);
int tc_square_grouped_pairs(cdl_ctx* ctx, const TcGroup* host_first, const TcGroup* dgroups,
                            const uint32_t* dtiles, int ntiles, double flops);
// Clusters of two the CTA-pair squaring can keep resident (0: unavailable).
int pair_clusters(cdl_ctx* ctx);
int tc_apply_grouped(cdl_ctx* ctx, const TcGroup* host_first, const TcGroup* dgroups, const uint32_t* dtiles,
                     int ntiles, int kp, int gate_mask, int kc, double work);
int apply_tc(cdl_ctx* ctx, const cdl_chain* ch, int level, const void* xop, float* partial,
             int k, int splits);
int apply_tc_mat(cdl_ctx* ctx, const void* amat, int np, const void* xop, float* partial, int kp,
                 int splits);
bool tc_supported(cdl_ctx* ctx);
// Anomalous edge set and per-node top edges (score.cu).
int cad_edges(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1, const double* Z2,
              const double* vol1, const double* vol2, int64_t n, int k, bool fp64, double delta, int64_t cap,
              const int64_t* nodes, int n_nodes, int m, int64_t* ij, double* val, int64_t* partner, double* pval,
              double* F, cdl_edge_result* res);

// Sparse scoring over the edges of changed nodes (score.cu).
int changed_nodes(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n, int T, int* list, int* count_dev);
int cad_score_changed(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1, const double* Z2,
                      const double* vol1, const double* vol2, int64_t n, int k, bool fp64, const int* changed,
                      int m, int topk, double* F, int64_t* top_idx);

// ---- batched form (one launch per step over many graphs) ----
// A device tile table: entries (b << 12) | g, or a kernel-specific packing.
struct BTiles {
  const uint32_t* p = nullptr;
  int count = 0;
};
// Graph build of one graph of a batch (device pointers).
struct GGraph {
  const double* X;  // n x T
  int* Xt;          // T x n fixed-point copy
  double* A;        // n x n
  double* D;        // n
  double* vol;
  double* sigma;
  void* sel;        // graph_select_bytes(): selection state and histogram
  int n, T;
};
size_t graph_select_bytes();
struct GraphTiles {
  std::vector<uint32_t> fixed;   // (b << 12) | g, 1024-sample blocks of X
  std::vector<uint32_t> dist;    // g | bi << 12 | bj << 22, 64-node blocks, bi <= bj
  std::vector<int4> sel;         // (g, first row, end row, 0): about 2^17 keys each
  std::vector<uint32_t> rows;    // (i << 12) | g
};
void graph_grouped_tiles(const std::vector<int>& n, int T, GraphTiles& out);
struct GraphBatch {
  int G2 = 0;
  double sigma = 0;              // <= 0: median rule per graph
  const GGraph* gs = nullptr;    // device
  void* sel_all = nullptr;       // the graphs' selection blocks, contiguous
  size_t sel_bytes = 0;
  BTiles fixed, dist, rows;
  const int4* sel = nullptr;
  int sel_count = 0;
  double dist_terms = 0, select_bytes = 0, kernel_bytes = 0;
};
int graph_build_grouped(cdl_ctx* ctx, const GraphBatch& b);

// Level-0 formation of one graph of a batch: bf16 chain with A kept as bf16
// hi/lo (the recursive update's operand) and as float hi/lo planes (the
// float-float residual's operand).
struct CGraph {
  const double* A;   // n x n
  const double* D;   // npad, zero padded
  const double* vol;
  double* rsd;       // npad: D^{-1/2}
  double* u;         // npad
  float* rsf;        // npad
  float* uf;         // npad
  uint16_t* aslices; // bf16 6 npad x npad: the exact slices of A (weights at most 1)
  void* L0;          // bf16 npad x npad
  void* aop;         // bf16 2 npad x npad: A_hi, A_lo
  int n, npad;
};
// Tile tables: vec (b << 12) | g over npad / 256 blocks; init (b << 12) | g
// over 2048-group blocks of npad^2 / 8 (level 0, A hi/lo and A's six exact
// slices).
int chain_init_grouped(cdl_ctx* ctx, const CGraph* cg, BTiles vec, BTiles init, double bytes);

// Projection of one graph of a batch.
struct PGraph {
  const double* A;
  double* Y;
  double* part;   // ceil(n / 256) x k column partial sums
  int n, pad;
};
int project_rows_per_block(int k);
// blocks: (b << 12) | g over ceil(n / rows_per_block); chunks: 256-row
// chunks; elem: 256-element blocks of n x k.
int project_grouped(cdl_ctx* ctx, const PGraph* gs, int G2, BTiles blocks, int rpb, int k, uint64_t seed,
                    BTiles chunks, BTiles elem, double adds);

// Solve commands, per graph, set by the decision kernel after each step.
enum { CMD_STEP = 1, CMD_FULL = 2, CMD_RECUR = 4 };

// Buffers of one graph of a batch (device pointers; n x k row-major blocks,
// npad-padded operands as in the single-graph solve).
struct BGraph {
  int n, np;
  int res_tiles;    // blocks whose partial sums a full residual leaves in red (= elem_blocks)
  int elem_blocks;  // 256-element blocks of n x k
  int kg;           // Z slice rows (k rounded up to 32)
  int pad0;
  const double* D;
  const double* rsd;
  const double* vol;
  unsigned long long* zmax;   // k: bits of max |Z| per column
  double* zc;                 // k: the column scales (powers of two)
  void* zs;                   // bf16 6 kg x npad: the exact slices of Z / c, transposed
  const double* Gp;           // RESID_PAIRS planes npad x kg of A Z
  const double* Y;
  double* Z;
  double* R;
  float* x;
  void* xop;        // bf16 2kp x npad
  float* part;      // npad x 2kp
  float* part2;
  float* dz;        // npad x kp
  void* dzop;       // bf16 2kp x npad
  double* red;      // elem_blocks
  double* cs;       // ceil(n / 256) x k
};

// Refinement state of one graph, on the device.
struct BState {
  int cmd;
  int iters;
  int exact;
  int pad;
  double yy, rel, drift;
  double hist[64];
};


struct BatchSolve {
  int G2 = 0, k = 0, kp = 0, d = 0, max_slots = 0, max_iter = 0;
  double rel_tol = 0;
  bool always_full = false;
  const BGraph* gs = nullptr;
  BState* st = nullptr;
  int* active = nullptr;                 // device: graphs still running after the last slot
  BTiles t32, elem, cs, apply;
  BTiles zst;                            // (b << 12) | g over 256-element blocks of kg x npad
  BTiles runits;                         // g | row tile << 16 over the 128-row tiles of every graph
  const ResidGroup* rgroups = nullptr;   // device, G2
  unsigned long long* zmax_all = nullptr;   // every graph's zmax, contiguous
  size_t zmax_bytes = 0;
  int kg = 0;
  double resid_work = 0;                 // flops of one full exact residual of every graph
  const TcGroup* lvl_groups = nullptr;   // device, d arrays of G2 (level-major)
  const TcGroup* lvl_first = nullptr;    // host, entry 0 of each level array
  const TcGroup* res_groups = nullptr;   // device, A_hi then A_lo arrays of G2
  const TcGroup* res_first = nullptr;    // host, 2 entries
  double apply_bytes = 0;                // per grouped level apply
};
// R = Y, Z = 0, ||Y|| and the first command of every graph.
int batch_solve_start(cdl_ctx* ctx, const BatchSolve& b);
// One refinement slot (a step or a certification per graph that has not
// stopped); *b.active counts the graphs still running after it.
int batch_solve_slot(cdl_ctx* ctx, const BatchSolve& b);
// Tile of the batched exact residual for k right-hand sides: 128 rows x kg.
void batch_residual_tile(int k, int* tm, int* tn);

// One pair of a batch for the grouped scoring launches.
struct ScoreJob {
  const double* A1;
  const double* A2;
  const double* Z1;
  const double* Z2;
  const double* vol1;
  const double* vol2;
  void* ab;         // 16 n k bytes
  double* contrib;  // ceil(n / 64) x n
  double* F;
  int64_t* top;
  unsigned* cmax;   // 2k column bounds (float32 scoring)
  int n;
  int pad;
};
// elem: (b << 12) | p over n k / 256 blocks; pairs: p | bi << 12 | bj << 22
// (64-node blocks, bi <= bj); nodes: (b << 12) | p over n / 256 blocks.
// cmax_all: the G x 2k column bounds the jobs point into (one block).
int cad_score_grouped(cdl_ctx* ctx, const ScoreJob* jobs, int G, int k, bool fp64, int topk, BTiles elem,
                      BTiles pairs, BTiles nodes, double bytes, unsigned* cmax_all);

// ---- graphs regenerated in row panels (larger than device memory) ----
// A Gaussian-kernel graph kept only as its node series (graph.cu): exact
// distances of grid inputs from three bf16 digit planes, sigma, degrees.
struct RegenGraph {
  int id = 0;                       // workspace tag (the graphs of a pair: 0, 1)
  const double* X = nullptr;        // n x T, on the 2^-16 grid
  int n = 0, T = 0, rows = 0, tp = 0;
  const void* planes = nullptr;     // three bf16 digit planes, rows x tp
  const long long* norms = nullptr; // |a_i|^2
  const int* offgrid = nullptr;     // bit 0: input off the grid
  double* sigma = nullptr;          // device
  double* D = nullptr;              // device n (the caller's)
  double* vol = nullptr;            // device 1 (the caller's)
};
// Planes, norms, sigma (lower median unless sigma > 0), D and vol; `panel`
// is P x n float64 scratch.
int graph_regen_init(cdl_ctx* ctx, RegenGraph& g, const double* X, int64_t n, int T, double sigma, double* panel,
                     int P);
// Rows r0 .. r0 + rows - 1 of A into panel (A[(i - r0) n + j]), their
// degrees into D[i] (r0 a multiple of 128, rows <= the panel's rows).
int regen_panel(cdl_ctx* ctx, const RegenGraph& g, double* panel, int r0, int rows, double* D);
// What the solve needs to form A Z of such a graph.
struct RegenSource {
  const RegenGraph* g = nullptr;
  double* panel = nullptr;          // P x n float64
  void* slicesT = nullptr;          // 6 x npad x P bf16 (transposed exact slices of a panel)
  double* Dscratch = nullptr;       // n (degrees recomputed by each regeneration)
  int P = 0;
};
// tc_gemm.cu: squared distances of a panel (rows row0 .. row0 + prows - 1,
// multiples of 128) into panel[(i - row0) n + j]: whole rows, or (upper)
// only the tiles of the upper block triangle.
int dist_tc_panel(cdl_ctx* ctx, const void* planes, const long long* norms, int n, int rows, int tp, double* panel,
                  int row0, int prows, bool upper, const int* offgrid);
// G (RESID_PAIRS planes npad x kp, as for resid_tc) += the pair products of
// A[:, c0 .. c0 + Pk) Z[c0 .. c0 + Pk) from the transposed exact slices of
// the panel (6 planes npad x Pw, Pk <= Pw columns in use, multiples of 256)
// and Z / c's slices (6 planes kp x npad).
int resid_tc_panel(cdl_ctx* ctx, const void* slicesT, int np, int Pw, int Pk, int c0, const void* zslices, int kp,
                   double* G);
// Score tiles tile0 .. tile1 - 1 of the upper-triangle numbering (tile1 < 0:
// all), A1 and A2 holding rows row0 .. (A[(i - row0) n + j]).
int score_tc_tiles(cdl_ctx* ctx, const void* uplanes, const void* vplanes, const long long* dint,
                   const double* oscale, int n, int rows, int k2p, const double* A1, const double* A2, int row0,
                   long long tile0, long long tile1, double* contrib);
// chain.cu: chain vectors from ch->D and ch->vol; level-0 rows from a panel;
// the panel's transposed exact slices.
int chain_vectors_only(cdl_ctx* ctx, cdl_chain* ch);
int chain_level0_panel(cdl_ctx* ctx, cdl_chain* ch, void* L0, const double* panel, int r0, int rows);
int panel_slices_t(cdl_ctx* ctx, const double* panel, int n, int np, int r0, int rows, int Pw, void* slicesT);
// project.cu: rows r0 .. r0 + rows - 1 of Y from a panel; column centring.
int project_panel(cdl_ctx* ctx, const double* panel, int64_t n, int r0, int rows, int k, uint64_t seed, double* Y,
                  const unsigned long long* amax_bits);
int project_center(cdl_ctx* ctx, int64_t n, int k, double* Y);
// score.cu: CAD scores (bf16 tensor-core Gram) with A1 and A2 supplied row
// panel by row panel: fill(r0, rows, &A1, &A2) makes rows r0 .. r0 + rows - 1
// of both graphs available.
int cad_score_panels(cdl_ctx* ctx, const double* Z1, const double* Z2, const double* vol1, const double* vol2,
                     int64_t n, int k, int P,
                     const std::function<int(int r0, int rows, const double** A1, const double** A2)>& fill, int topk,
                     double* F, int64_t* top_idx);
// regen.cu: the whole pair with graphs regenerated in row panels.
int pair_regen(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n, int T, const cdl_pair_opts* o,
               double* F, int64_t* top_idx, cdl_solve_stats* stats1, cdl_solve_stats* stats2);
// api.cu: a bf16 chain for graphs given by panels (no A operands), levels
// 0 .. resident - 1 on the device, the rest in pinned host memory.
int chain_create_regen(cdl_ctx* ctx, int64_t n, int d, int resident, cdl_chain** out);

// solve.cu
int chain_solve(cdl_ctx* ctx, const cdl_chain* ch, const double* A, const double* Y, int k,
                const cdl_solve_opts* opts, double* Z, cdl_solve_stats* stats);
// project.cu
// amax_bits (device, optional): the float64 bits of max |A| if already known
// (nullptr: found by a pass over A).
int project(cdl_ctx* ctx, const double* A, int64_t n, int k, uint64_t seed, double* Y,
            const unsigned long long* amax_bits = nullptr);
// score.cu
int cad_score(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1,
              const double* Z2, const double* vol1, const double* vol2, int64_t n, int k,
              cdl_dtype score_dtype, int topk, double* F, int64_t* top_idx);

}  // namespace cdl
