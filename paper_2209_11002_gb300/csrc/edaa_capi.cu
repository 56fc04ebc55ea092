// Host side of the EDAA C ABI (include/edaa.h): argument checks, device
// memory, launch shapes, CUDA-graph capture, Algorithm 2's selection rule.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <atomic>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/edaa.h"
#include "edaa_internal.cuh"
#include "edaa_tc.cuh"

using namespace edaa;

namespace {

thread_local std::string g_err;

edaa_status fail(edaa_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

edaa_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? EDAA_ERR_OOM : EDAA_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

// Failure injection for tests of the out-of-memory path: when the counter is
// k >= 0, the k-th device allocation from then on fails with
// cudaErrorMemoryAllocation without calling the runtime (-1: off).
std::atomic<int> g_fail_alloc{-1};

bool alloc_fails() {
  int k = g_fail_alloc.load();
  while (k >= 0) {
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 0;
  }
  return false;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (alloc_fails()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  if (alloc_fails()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, s);
}

// NVTX range for the duration of a scope (the library's entry points), so
// that a profiler timeline shows which call enqueued which launches
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

#define CK(call, what)                          \
  do {                                          \
    cudaError_t e__ = (call);                   \
    if (e__ != cudaSuccess) return cuda_fail(e__, what); \
  } while (0)

struct TileCfg {
  int Rm, WP1, SPT, WP2;
};

// Register-tile limits of the compiled kernels (must match PassTraits): the
// default slot shape (up to spt_max pixels x rq1_max runs per thread) and,
// for p >= 3, the four-pixel shape (4 pixels x 1 run).
int rq1_max(int p) { return p <= 2 ? 4 : (p <= 4 ? 2 : 1); }
int spt_max(int p) { return p <= 4 ? 2 : 1; }
int rq2_max(int p) { return p <= 2 ? 4 : (p <= 4 ? 2 : 1); }

bool tile_ok(const TileCfg& t, int L, int p, int M) {
  if (t.Rm < 1 || t.Rm > M) return false;
  const bool four = t.SPT == 4 && p >= 3;
  if (8 % t.WP1 || 8 % t.WP2 || t.SPT < 1 || (!four && t.SPT > spt_max(p))) return false;
  const int WR1 = 8 / t.WP1, WR2 = 8 / t.WP2;
  if ((t.Rm + WR1 - 1) / WR1 > (four ? 1 : rq1_max(p))) return false;
  if ((t.Rm + WR2 - 1) / WR2 > rq2_max(p)) return false;
  const int Nt = 32 * t.WP1 * t.SPT;
  const PassSmem s = pass_smem(L, padded_ld(L), round_up(L, 4), p, t.Rm, Nt);
  return (size_t)s.total * 4 <= 200 * 1024;
}

size_t tile_smem(const TileCfg& t, int L, int p) {
  const int Nt = 32 * t.WP1 * t.SPT;
  return (size_t)pass_smem(L, padded_ld(L), round_up(L, 4), p, t.Rm, Nt).total * 4;
}

// Default launch shape: the largest run group the register tiles allow with
// both phases' warps busy, a pixel tile of 64, and 2 CTAs per SM of shared
// memory where it fits.
TileCfg default_tile(int L, int p, int M) {
  std::vector<TileCfg> cands;
  for (int Rm : {8, 6, 4, 3, 2, 1}) {
    if (Rm > M) continue;
    for (int WP1 : {2, 1, 4, 8})
      for (int WP2 : {1, 2, 4, 8}) {
        TileCfg t{Rm, WP1, 64 / (32 * WP1) > 0 ? std::max(1, 64 / (32 * WP1)) : 1, WP2};
        if (32 * WP1 * t.SPT != 64) continue;
        if (tile_ok(t, L, p, M)) cands.push_back(t);
      }
  }
  // score: busy warps in each phase (runs spread over warps), then bigger Rm
  auto score = [&](const TileCfg& t) {
    const int WR1 = 8 / t.WP1, WR2 = 8 / t.WP2;
    const double b1 = (double)t.Rm / (WR1 * ((t.Rm + WR1 - 1) / WR1));
    const double b2 = (double)t.Rm / (WR2 * ((t.Rm + WR2 - 1) / WR2));
    const int RG = (M + t.Rm - 1) / t.Rm;
    const double brun = (double)M / (RG * t.Rm);
    return b1 * b2 * brun * (1.0 + 0.01 * t.Rm) * (tile_smem(t, L, p) <= 110 * 1024 ? 1.0 : 0.8);
  };
  TileCfg best{1, 2, 1, 8};
  double bs = -1.0;
  for (const auto& t : cands) {
    const double s = score(t);
    if (s > bs) { bs = s; best = t; }
  }
  return best;
}

std::vector<TileCfg> tile_candidates(int L, int p, int M) {
  std::vector<TileCfg> out;
  for (int Rm : {1, 2, 3, 4, 5, 6, 8, 10, 12, 16})
    for (int WP1 : {1, 2, 4, 8})
      for (int SPT : {1, 2, 4})
        for (int WP2 : {1, 2, 4, 8}) {
          TileCfg t{Rm, WP1, SPT, WP2};
          const int Nt = 32 * WP1 * SPT;
          if (Nt < 32 || Nt > 128) continue;
          if (tile_ok(t, L, p, M)) out.push_back(t);
        }
  return out;
}

std::map<std::tuple<int, int, int, int, int>, TileCfg>& tune_cache() {
  static std::map<std::tuple<int, int, int, int, int>, TileCfg> c;
  return c;
}

}  // namespace

namespace edaa {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace edaa

struct CubeHost {
  int L, N, p, M, Ls, Lr, Mp;
  int hist_cap = 0;  // rows of the loss log (T with record_loss, else 0)
  TileCfg tile;
  bool tile_fixed = false;  // set by the caller (edaa_config.tile): not autotuned
  int RG, Pg, Nt, ntiles, lchunk, nlchunk;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  float* X_in = nullptr;  // N x L staging copy of the caller's X
  double* bsum = nullptr; // per-block band sums for the mean pixel
  double* scale = nullptr; // per-pixel 1/||x_i|| (FP64)
  // tensor-core path
  int tc = 0, esz = 4, kp = 0, Npad = 0;
  int tc_rg = 0;           // run groups of a tensor-core cube (0: the fewest the TMEM allows)
  int tc_rm_fixed = 0;     // runs per group set by the caller (edaa_config.tile[0])
  void* Xk = nullptr;      // N x kp compute-type copy of the centred X (pixel-major)
  void* XT = nullptr;      // (L+1) x Npad band-major copy
  CUtensorMap* tmaps = nullptr;  // device, 4 maps
  CubeDev dev;
  std::vector<uint64_t> seeds;
  std::vector<double> gammas;
};

struct edaa_ctx {
  edaa_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, sm_count = 0, blocks_per_sm = 1;
  std::vector<CubeHost> cubes;
  Batch hb;
  Batch* d_batch = nullptr;
  int* d_status = nullptr;
  unsigned* d_bar = nullptr;
  unsigned long long* d_trace = nullptr;  // phase trace: 3 x kTraceCap starts, then 3 x kTraceCap ends
  int trace_n[3] = {0, 0, 0};             // phases of the last sequence of each mode
  size_t smem = 0;
  int grid = 0;
  int outer_done = 0;
  bool broken = false;
  cudaGraphExec_t g_solve = nullptr;
  int g_solve_n = -1;
  bool graphs_ok = true;
  int graph_state = 0;  // 1: the last edaa_solve replayed its captured graph; -1: capture failed; 0: no solve yet
  int launches_last_solve = 0;
};

static edaa_status check_status(edaa_ctx* c) {
  if (c->broken) return fail(EDAA_ERR_STATE, "context is unusable after an earlier device error");
  return EDAA_OK;
}

// Tensor-core cubes: 128-pixel tiles; the largest run group whose padded
// column count Rgp fits TMEM next to one accumulator per 128-band tile
// (Rgp * (1 + band tiles) <= 512 columns, Rgp <= 256), balanced over groups.
static void tc_tile(CubeHost& h) {
  const int rgp_max = tc_rgp_max(h.L, h.esz, h.tc == 3, h.p);
  const int rm_max = std::max(1, std::min({128, rgp_max / h.p, 2048 / (h.p * h.p)}));
  const int RG = std::min(h.M, std::max((h.M + rm_max - 1) / rm_max, h.tc_rg));
  h.tile.Rm = h.tile_fixed ? std::min(h.tc_rm_fixed, rm_max) : (h.M + RG - 1) / RG;
  h.tile.WP1 = 4;  // the CUDA-core fit pass runs on the same 128-pixel tiles
  h.tile.SPT = 1;
  h.tile.WP2 = 1;
}

// Assign pass work items (run group x pixel group) and merge work items.
static void plan(edaa_ctx* c) {
  const int G = c->sm_count * c->blocks_per_sm;
  double total = 0.0;
  for (auto& h : c->cubes) total += (double)h.N * h.L * h.M * h.p;
  int cta = 0, unit = 0, run0 = 0;
  int units_total = 0;
  for (auto& h : c->cubes) units_total += h.M;
  for (auto& h : c->cubes) {
    if (h.tc) tc_tile(h);
    h.Nt = 32 * h.tile.WP1 * h.tile.SPT;
    h.ntiles = (h.N + h.Nt - 1) / h.Nt;
    h.RG = (h.M + h.tile.Rm - 1) / h.tile.Rm;
    const double share = total > 0 ? (double)h.N * h.L * h.M * h.p / total : 1.0;
    int n = std::max(h.RG, (int)floor(share * G));
    h.Pg = std::max(1, std::min(h.ntiles, n / h.RG));
    // even tiles per pixel group
    const int per = (h.ntiles + h.Pg - 1) / h.Pg;
    h.Pg = (h.ntiles + per - 1) / per;
    // merge chunks: aim for about G units in total
    // merge units (run x band chunk): one wave over the grid where possible
    const int want = std::max(1, G / std::max(1, units_total));
    const int lch = std::max(1, (h.L + want - 1) / want);
    h.lchunk = lch;
    h.nlchunk = (h.L + lch - 1) / lch;
    // the B-merge keeps Pg x p scale factors in shared memory
    const int pg_fit = (int)(((long long)(c->smem / 8) - merge_smem(lch, h.p, 0).total) / h.p);
    if (h.Pg > pg_fit) h.Pg = std::max(1, pg_fit);
    CubeDev& d = h.dev;
    d.L = h.L; d.Ls = h.Ls; d.Lr = h.Lr; d.N = h.N; d.p = h.p; d.M = h.M; d.Mp = h.Mp;
    d.Nst = round_up(h.N, 32);
    d.logN = log((double)h.N);
    d.LT = (h.L + 1 + 31) / 32;
    d.Rm = h.tile.Rm; d.RG = h.RG; d.Pg = h.Pg; d.Nt = h.Nt; d.WP1 = h.tile.WP1; d.SPT = h.tile.SPT;
    d.WP2 = h.tile.WP2; d.ntiles = h.ntiles;
    d.tc = h.tc;
    d.tc_kp = h.kp;
    d.tc_nbt = (h.L + 1 + 127) / 128;
    d.tc_nkc = h.tc ? (h.L + (128 / h.esz) - 1) / (128 / h.esz) : 0;
    d.tc_rgp = h.tc ? round_up(h.tile.Rm * h.p, 16) : 0;
    d.cta0 = cta; d.lchunk = h.lchunk; d.nlchunk = h.nlchunk; d.unit0 = unit; d.run0 = run0;
    cta += h.RG * h.Pg;
    unit += h.M * h.nlchunk;
    run0 += h.M;
  }
  c->hb.pass_items = cta;
  c->hb.merge_units = unit;
  c->hb.total_runs = run0;
  c->grid = std::min(G, std::max(cta, unit));
  if (c->grid < 1) c->grid = 1;
}

// shared memory of the pass and fit work items of a cube (no merge terms)
static size_t pass_item_smem(const CubeHost& h) {
  size_t s = tile_smem(h.tile, h.L, h.p);
  if (h.tc) {
    const int rb = std::min(h.tile.Rm, (8 / h.tile.WP1) * rq1_max(h.p));
    s = (size_t)pass_smem(h.L, h.Ls, h.Lr, h.p, rb, 128).total * 4;  // fit pass in run blocks
    const int rgp = round_up(h.tile.Rm * h.p, 16);  // the widest group this cube can take (smaller ones need less)
    s = std::max(s, (size_t)tc_smem_max(rgp, h.esz, h.tc == 3, h.p, h.L, kTcSmemCap));
  }
  return s;
}

static size_t cube_smem(const CubeHost& h) {
  size_t s = pass_item_smem(h);
  return std::max(s, (size_t)merge_smem(h.lchunk, h.p, h.Pg).total * 8);
}

// Partial buffers are sized for the largest pixel-group count a plan can use.
static size_t arena_layout(CubeHost& h, int Pg_cap, bool assign) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    const size_t o = off;
    off += bytes;
    return o;
  };
  const size_t N = h.N, L = h.L, Mp = h.Mp, M = h.M, p = h.p, Ls = h.Ls;
  const size_t Nst = round_up(h.N, 32);  // state rows: one run column over the pixels
  const size_t tcb = h.tc ? 1 : 0, parts = h.tc == 3 ? 2 : 1;  // split operands: high and low copies
  // tensor-core cubes keep no B logits (regenerated from the RNG, S and Lambda)
  size_t oX = take(N * Ls * 4), oXin = take(N * L * 4), oA = take(Nst * Mp * 4), oB = take((1 - tcb) * Nst * Mp * 4);
  size_t oEf = take(L * Mp * 4), oEd = take(L * Mp * 8), oRf = take(L * Mp * 4), oXAt = take(L * Mp * 8);
  size_t oAAt = take(M * p * p * 8), olse = take(Mp * 4), oe1 = take(M * 4), oe2 = take(M * 4);
  size_t oe1d = take(M * 8), oe2d = take(M * 8), osig = take(M * 8);
  size_t opart = take((size_t)Pg_cap * (L + 1) * Mp * 4), opmax = take((size_t)Pg_cap * Mp * 4);
  size_t opaa = take((size_t)Pg_cap * M * p * p * 4), opfit = take((size_t)Pg_cap * M * 3 * 8);
  size_t ofit = take(M * 8), ofitmax = take(M * 8), oloss = take(M * 8), omu = take(M * 8);
  size_t ohist = take((size_t)h.hist_cap * M * 8);
  size_t oseeds = take(M * 8), ogam = take(M * 8);
  size_t orho = take(L * Mp * 8), obref = take(Mp * 4);  // nlchunk <= L band chunks
  size_t ogpart = take(L * M * p * p * 8);
  // the band-major copy of X only for TF32 (BF16 passes read the pixel-major tiles both ways)
  const size_t xtb = (h.tc == 1 || h.tc == 3) ? 1 : 0;
  size_t oXk = take(tcb * parts * N * h.kp * h.esz), oXT = take(xtb * parts * (L + 1) * h.Npad * h.esz);
  size_t opE = take(tcb * parts * Mp * h.kp * h.esz), opS = take(tcb * 2 * Mp * h.kp * h.esz);
  size_t oSd = take(tcb * L * Mp * 8), oRd = take(tcb * L * Mp * 8), olam = take(tcb * Mp * 8);
  size_t or16 = take(tcb * Nst * Mp * 2);
  size_t otm = take(tcb * TM_COUNT * 128);
  size_t oscale = take(N * 8), oxbar = take(L * 8), osx = take((L + 1) * 8), obsum = take((size_t)normalize_blocks(h.N) * L * 8);
  if (assign) {
    char* b = (char*)h.arena;
    CubeDev& d = h.dev;
    d.X = (float*)(b + oX);
    h.X_in = (float*)(b + oXin);
    d.logA = (float*)(b + oA);
    d.logB = h.tc ? nullptr : (float*)(b + oB);
    d.Ef = (float*)(b + oEf);
    d.Ed = (double*)(b + oEd);
    d.Rf = (float*)(b + oRf);
    d.XAt = (double*)(b + oXAt);
    d.AAt = (double*)(b + oAAt);
    d.lse = (float*)(b + olse);
    d.eta1 = (float*)(b + oe1);
    d.eta2 = (float*)(b + oe2);
    d.eta1d = (double*)(b + oe1d);
    d.eta2d = (double*)(b + oe2d);
    d.sig2 = (double*)(b + osig);
    d.part = (float*)(b + opart);
    d.pmax = (float*)(b + opmax);
    d.paa = (float*)(b + opaa);
    d.pfit = (double*)(b + opfit);
    d.fit = (double*)(b + ofit);
    d.fitmax = (double*)(b + ofitmax);
    d.loss2 = (double*)(b + oloss);
    d.mu = (double*)(b + omu);
    d.loss_hist = (double*)(b + ohist);
    d.seeds = (const uint64_t*)(b + oseeds);
    d.gammas = (const double*)(b + ogam);
    d.rho = (double*)(b + orho);
    d.bref = (int*)(b + obref);
    d.gpart = (double*)(b + ogpart);
    d.xbar = (double*)(b + oxbar);
    d.sx = (double*)(b + osx);
    h.bsum = (double*)(b + obsum);
    h.scale = (double*)(b + oscale);
    if (h.tc) {
      h.Xk = b + oXk;
      h.XT = xtb ? b + oXT : nullptr;
      d.Xk = h.Xk;
      d.panelE = b + opE;
      d.panelS = b + opS;
      d.Sd = (double*)(b + oSd);
      d.Rd = (double*)(b + oRd);
      d.lamd = (double*)(b + olam);
      d.r16 = (uint16_t*)(b + or16);
      h.tmaps = (CUtensorMap*)(b + otm);
      d.tmaps = h.tmaps;
    }
  }
  return off;
}

static edaa_status upload_x(edaa_ctx* c, CubeHost& h, const float* X) {
  CK(cudaMemcpyAsync(h.X_in, X, (size_t)h.N * h.L * 4, cudaMemcpyDefault, c->stream), "copy X");
  if (h.tc) {
    const edaa_status st = [&]() -> edaa_status {
      CK(launch_normalize(h.X_in, h.dev.X, h.scale, h.bsum, h.dev.xbar, h.dev.sx, h.L, h.Ls, h.N, c->cfg.normalize,
                          c->cfg.center, c->stream), "normalize");
      CK(launch_tc_prepare(h.dev, h.Xk, h.XT, h.Npad, c->stream), "tensor-core copies of X");
      return EDAA_OK;
    }();
    return st;
  }
  CK(launch_normalize(h.X_in, h.dev.X, h.scale, h.bsum, h.dev.xbar, h.dev.sx, h.L, h.Ls, h.N, c->cfg.normalize,
                      c->cfg.center, c->stream), "normalize");
  return EDAA_OK;
}

// TMA descriptors (128-byte swizzle, K-major boxes) for the tensor-core passes
static edaa_status make_tmaps(edaa_ctx* c, CubeHost& h) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        !fn)
      return fail(EDAA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const CUtensorMapDataType dt = h.esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint32_t kch = 128 / h.esz, es[2] = {1, 1};
  const int rgp = round_up(h.tile.Rm * h.p, 16);
  // the operand maps (128-byte swizzle, K-major boxes), in TcMap order; with
  // split operands the low parts follow the high parts in memory
  CUtensorMap m[TM_COUNT];
  memset(m, 0, sizeof m);
  const size_t nXk = (size_t)h.N * h.kp * h.esz, nXT = (size_t)(h.L + 1) * h.Npad * h.esz;
  const size_t nP = (size_t)h.Mp * h.kp * h.esz;
  struct Spec { void* ptr; cuuint64_t inner, outer; cuuint32_t box_outer; bool used; } spec[TM_STATE] = {
      {h.Xk, (cuuint64_t)h.kp, (cuuint64_t)h.N, 128, true},
      {h.XT, (cuuint64_t)h.Npad, (cuuint64_t)(h.L + 1), 128, h.tc != 2},
      {h.dev.panelE, (cuuint64_t)h.kp, (cuuint64_t)h.Mp, (cuuint32_t)rgp, true},
      {h.dev.panelS, (cuuint64_t)h.kp, (cuuint64_t)h.Mp, (cuuint32_t)rgp, true},
      {(char*)h.Xk + nXk, (cuuint64_t)h.kp, (cuuint64_t)h.N, 128, h.tc == 3},
      {(char*)h.XT + nXT, (cuuint64_t)h.Npad, (cuuint64_t)(h.L + 1), 128, h.tc == 3},
      {(char*)h.dev.panelE + nP, (cuuint64_t)h.kp, (cuuint64_t)h.Mp, (cuuint32_t)rgp, h.tc == 3},
      {(char*)h.dev.panelS + nP, (cuuint64_t)h.kp, (cuuint64_t)h.Mp, (cuuint32_t)rgp, true}};
  for (int i = 0; i < TM_STATE; ++i) {
    if (!spec[i].used) continue;
    const cuuint64_t dims[2] = {spec[i].inner, spec[i].outer};
    const cuuint64_t strides[1] = {spec[i].inner * (cuuint64_t)h.esz};
    const cuuint32_t box[2] = {kch, spec[i].box_outer};
    const CUresult r = enc(&m[i], dt, 2, spec[i].ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(EDAA_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  }
  {  // the log-abundance state, float32 Mp x Nst: boxes of 128 pixels x one run group's rows, unswizzled
    const int Nst = round_up(h.N, 32);
    const cuuint64_t dims[2] = {(cuuint64_t)Nst, (cuuint64_t)h.Mp};
    const cuuint64_t strides[1] = {(cuuint64_t)Nst * 4};
    const cuuint32_t box[2] = {128, (cuuint32_t)(h.tile.Rm * h.p)};
    const CUresult r = enc(&m[TM_STATE], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.dev.logA, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(EDAA_ERR_CUDA, "cuTensorMapEncodeTiled failed (state map)");
    const cuuint64_t strides16[1] = {(cuuint64_t)Nst * 2};
    const CUresult r2 = enc(&m[TM_R16], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, h.dev.r16, dims, strides16, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r2 != CUDA_SUCCESS) return fail(EDAA_ERR_CUDA, "cuTensorMapEncodeTiled failed (uniforms map)");
  }
  const int nmaps = TM_COUNT;
  CK(cudaMemcpyAsync(h.tmaps, m, nmaps * sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream),
     "upload tensor maps");
  return EDAA_OK;
}

// The device regions that hold a cube's iteration state (everything a later
// outer iteration reads), for checkpoints: pointers into the arena and sizes.
struct StateRegion {
  void* ptr;
  size_t bytes;
};
static std::vector<StateRegion> state_regions(const CubeHost& h) {
  const CubeDev& d = h.dev;
  const size_t L = h.L, Mp = h.Mp, M = h.M, p = h.p, Nst = round_up(h.N, 32);
  std::vector<StateRegion> r = {{d.logA, Nst * Mp * 4}, {d.Ef, L * Mp * 4}, {d.Ed, L * Mp * 8},
                                {d.Rf, L * Mp * 4},     {d.XAt, L * Mp * 8}, {d.AAt, M * p * p * 8},
                                {d.lse, Mp * 4},        {d.eta1, M * 4},    {d.eta2, M * 4},
                                {d.eta1d, M * 8},       {d.eta2d, M * 8},   {d.sig2, M * 8},
                                {d.rho, L * Mp * 8},    {d.bref, Mp * 4},   {d.gpart, L * M * p * p * 8},
                                {d.fit, M * 8},         {d.fitmax, M * 8},  {d.loss2, M * 8},
                                {d.mu, M * 8}};
  if (h.hist_cap > 0) r.push_back({d.loss_hist, (size_t)h.hist_cap * M * 8});
  if (h.tc) {
    const size_t parts = h.tc == 3 ? 2 : 1;
    r.push_back({d.panelE, parts * Mp * h.kp * h.esz});
    r.push_back({d.panelS, 2 * Mp * h.kp * h.esz});
    r.push_back({d.Sd, L * Mp * 8});
    r.push_back({d.Rd, L * Mp * 8});
    r.push_back({d.lamd, Mp * 8});
  } else {
    r.push_back({d.logB, Nst * Mp * 4});
  }
  return r;
}

// checkpoint layout: header, then per cube its layout key and the FP64 band
// sums of its X (sx, L + 1 values: a fingerprint of the data), then the
// regions in state_regions order
struct CkptHeader {
  char magic[8];
  int version, n_cubes, outer_done, record_loss, hist_cap, pad;
  uint64_t payload;
};
struct CkptCube {
  int L, N, p, M, tc, esz, kp, pad;
};

static edaa_status push_batch(edaa_ctx* c) {
  for (size_t i = 0; i < c->cubes.size(); ++i) c->hb.c[i] = c->cubes[i].dev;
  CK(cudaMemcpyAsync(c->d_batch, &c->hb, sizeof(Batch), cudaMemcpyHostToDevice, c->stream), "upload batch");
  return EDAA_OK;
}

// Enqueue one program (a sequence of phases) either as one persistent
// launch or as one launch per phase.
static edaa_status enqueue(edaa_ctx* c, int mode, int n_outer, int* launches) {
  const int nph = program_phase_count(mode, n_outer, c->cfg.K2, c->hb.record_loss);
  if (nph <= 0) return EDAA_OK;
  if (c->d_trace) {
    const size_t n = (size_t)std::min(nph, kTraceCap);
    CK(cudaMemsetAsync(c->d_trace + (size_t)mode * kTraceCap, 0xFF, n * 8, c->stream), "reset trace");
    CK(cudaMemsetAsync(c->d_trace + (size_t)(3 + mode) * kTraceCap, 0, n * 8, c->stream), "reset trace");
    c->trace_n[mode] = (int)n;
  }
  if (c->cfg.persistent && nph > 1) {
    CK(launch_program(c->d_batch, mode, c->outer_done, 0, nph, c->grid, c->smem, true, c->stream),
       "persistent launch");
    if (launches) *launches += 1;
  } else {
    for (int s = 0; s < nph; ++s) {
      CK(launch_program(c->d_batch, mode, c->outer_done, s, s + 1, c->grid, c->smem, false, c->stream),
         "phase launch");
      if (launches) *launches += 1;
    }
  }
  return EDAA_OK;
}

static edaa_status run_init(edaa_ctx* c) {
  CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "reset status");
  CK(cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->stream), "reset barrier");
  for (auto& h : c->cubes) {
    CK(cudaMemsetAsync(h.dev.XAt, 0, (size_t)h.L * h.Mp * 8, c->stream), "zero");
    CK(cudaMemsetAsync(h.dev.AAt, 0, (size_t)h.M * h.p * h.p * 8, c->stream), "zero");
    if (h.tc) {  // S and Lambda start from B^0 (no B-step taken); the B^0 uniforms
      CK(cudaMemsetAsync(h.dev.Sd, 0, (size_t)h.L * h.Mp * 8, c->stream), "zero");
      CK(cudaMemsetAsync(h.dev.lamd, 0, (size_t)h.Mp * 8, c->stream), "zero");
      if (h.tc != 3) CK(launch_fill_r16(h.dev, c->stream), "B^0 uniforms");
    }
  }
  edaa_status st = enqueue(c, MODE_INIT, 0, nullptr);
  if (st != EDAA_OK) return st;
  c->outer_done = 0;
  return EDAA_OK;
}

static edaa_status sync_status(edaa_ctx* c) {
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  int st = 0;
  CK(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  if (st & kStatTimeout) {
    c->broken = true;
    char msg[160];
    snprintf(msg, sizeof msg, "a bounded wait timed out (status 0x%x: bit 0 grid barrier; bits 9-14 tensor-core "
             "pipeline stages and the A state tile)", st);
    return fail(EDAA_ERR_TIMEOUT, msg);
  }
  return EDAA_OK;
}

// Autotuner: time each candidate launch shape on this cube's data (one
// A-pass + merge and one B-pass + merge, as separate launches) and keep the
// fastest; results are cached per (device, L, N, p, M).
// Time of 2 outer iterations (one launch per phase, after a warm-up one) with
// the batch's current shapes.
static edaa_status time_candidate(edaa_ctx* c, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  edaa_status st = push_batch(c);
  if (st != EDAA_OK) return st;
  st = run_init(c);
  if (st != EDAA_OK) return st;
  const int persistent = c->cfg.persistent;
  c->cfg.persistent = 0;
  st = enqueue(c, MODE_OUTER, 1, nullptr);
  CK(cudaEventRecord(e0, c->stream), "event");
  if (st == EDAA_OK) st = enqueue(c, MODE_OUTER, 2, nullptr);
  CK(cudaEventRecord(e1, c->stream), "event");
  c->cfg.persistent = persistent;
  if (st != EDAA_OK) return st;
  CK(cudaEventSynchronize(e1), "event sync");
  CK(cudaEventElapsedTime(ms, e0, e1), "elapsed");
  return sync_status(c);  // a timed-out wait ends the tuning with an error rather than more waits
}

std::map<std::tuple<int, int, int, int, int, int>, int>& tc_tune_cache() {
  static std::map<std::tuple<int, int, int, int, int, int>, int> c;
  return c;
}

// CUDA-core cubes: the tile candidates.  Tensor-core cubes: the number of run
// groups, from the fewest the tensor memory allows up to three more (smaller
// groups give each pass more CTAs and shorter epilogues per tile).
static edaa_status autotune(edaa_ctx* c) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  edaa_status st = EDAA_OK;
  for (size_t ci = 0; ci < c->cubes.size() && st == EDAA_OK; ++ci) {
    CubeHost& h = c->cubes[ci];
    if (h.tile_fixed) continue;
    if (h.tc) {
      // the cube's tensor maps follow its run groups: rebuilt for each
      // candidate and for the one kept, before any other cube is timed
      auto key = std::make_tuple(c->device, h.L, h.N, h.p, h.M, h.tc);
      auto it = tc_tune_cache().find(key);
      if (it != tc_tune_cache().end()) {
        h.tc_rg = it->second;
        plan(c);
        st = make_tmaps(c, h);
        continue;
      }
      h.tc_rg = 0;
      tc_tile(h);
      const int rg0 = (h.M + h.tile.Rm - 1) / h.tile.Rm;
      int best = rg0, last_rm = 0;
      float best_ms = 1e30f;
      for (int rg = rg0; rg <= std::min(h.M, rg0 + 3) && st == EDAA_OK; ++rg) {
        h.tc_rg = rg;
        plan(c);
        if (h.tile.Rm == last_rm) continue;  // the same groups as a smaller count
        last_rm = h.tile.Rm;
        st = make_tmaps(c, h);
        float ms = 0.f;
        if (st == EDAA_OK) st = time_candidate(c, e0, e1, &ms);
        if (st == EDAA_OK && ms < best_ms) { best_ms = ms; best = rg; }
      }
      h.tc_rg = best;
      if (st == EDAA_OK) {
        tc_tune_cache()[key] = best;
        plan(c);
        st = make_tmaps(c, h);
      }
      continue;
    }
    auto key = std::make_tuple(c->device, h.L, h.N, h.p, h.M);
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      h.tile = it->second;
      continue;
    }
    std::vector<TileCfg> cands = tile_candidates(h.L, h.p, h.M);
    TileCfg best = h.tile;
    float best_ms = 1e30f;
    for (const auto& t : cands) {
      h.tile = t;
      plan(c);
      if (cube_smem(h) > c->smem) continue;
      float ms = 0.f;
      st = time_candidate(c, e0, e1, &ms);
      if (st != EDAA_OK) break;
      if (ms < best_ms) { best_ms = ms; best = t; }
    }
    h.tile = best;
    if (st == EDAA_OK) tune_cache()[key] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EDAA_OK) return st;
  plan(c);
  for (auto& h : c->cubes)
    if (h.tc) {
      st = make_tmaps(c, h);
      if (st != EDAA_OK) return st;
    }
  return push_batch(c);
}

extern "C" {

void edaa_config_default(edaa_config* cfg) {
  if (!cfg) return;
  cfg->T = 100;
  cfg->K1 = 5;
  cfg->K2 = 5;
  cfg->normalize = 1;
  cfg->precision = EDAA_FP32;
  cfg->fit_norm = 0;
  cfg->coherence = 0;
  cfg->fit_ratio = 1.05;
  cfg->persistent = 1;
  cfg->autotune = 0;
  cfg->barrier_timeout_ms = 2000.0;
  cfg->center = 1;
  cfg->trace = 0;
  for (int i = 0; i < 4; ++i) cfg->tile[i] = 0;
  cfg->record_loss = 0;
}

const char* edaa_last_error(void) { return g_err.c_str(); }

int edaa_select_rule(const double* fit, const double* mu, int M, double fit_ratio) {
  if (!fit || !mu || M < 1) return -1;
  int first = -1;
  double fmin = INFINITY;
  for (int m = 0; m < M; ++m)
    if (isfinite(fit[m]) && fit[m] < fmin) { fmin = fit[m]; first = m; }
  if (first < 0) return -1;
  int best = -1;
  for (int m = 0; m < M; ++m) {
    if (!isfinite(fit[m]) || !(fit[m] <= fit_ratio * fmin)) continue;
    if (best < 0 || mu[m] < mu[best]) best = m;
  }
  return best;
}

edaa_status edaa_init(edaa_ctx** out, const edaa_cube* cubes, int n_cubes, const edaa_config* cfg, void* stream) {
  NvtxRange nvtx_range("edaa_init");
  g_err.clear();
  if (!out) return fail(EDAA_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cubes || n_cubes < 1 || n_cubes > kMaxCubes) return fail(EDAA_ERR_ARG, "n_cubes must be 1..16");
  edaa_config conf;
  edaa_config_default(&conf);
  if (cfg) conf = *cfg;
  if (conf.T < 0 || conf.K1 < 0 || conf.K2 < 0) return fail(EDAA_ERR_ARG, "T, K1, K2 must be >= 0");
  if (!(conf.fit_ratio >= 1.0)) return fail(EDAA_ERR_ARG, "fit_ratio must be >= 1");
  if (conf.precision < EDAA_FP32 || conf.precision > EDAA_TF32X3) return fail(EDAA_ERR_ARG, "unknown precision");
  for (int i = 0; i < n_cubes; ++i) {
    const edaa_cube& q = cubes[i];
    if (!q.X) return fail(EDAA_ERR_ARG, "cube X is NULL");
    if (q.L < 1 || q.L > kMaxL) return fail(q.L < 1 ? EDAA_ERR_ARG : EDAA_ERR_UNSUPPORTED, "L must be 1..319");
    if (q.p < 1 || q.p > kMaxP) return fail(q.p < 1 ? EDAA_ERR_ARG : EDAA_ERR_UNSUPPORTED, "p must be 1..8");
    if (q.N < q.p) return fail(EDAA_ERR_ARG, "N must be >= p");
    if (q.M < 1) return fail(EDAA_ERR_ARG, "M must be >= 1");
    if (!q.seeds || !q.gammas) return fail(EDAA_ERR_ARG, "seeds and gammas are required");
    for (int m = 0; m < q.M; ++m)
      if (!(q.gammas[m] > 0.0) || !isfinite(q.gammas[m])) return fail(EDAA_ERR_ARG, "gammas must be finite and > 0");
    if (conf.tile[0] != 0) {
      const TileCfg t{conf.tile[0], conf.tile[1], conf.tile[2], conf.tile[3]};
      const bool tc = conf.precision != EDAA_FP32 && q.M * q.p >= 64;  // tensor-core cube: tile[0] alone
      const bool pos = t.Rm > 0 && t.WP1 > 0 && t.SPT > 0 && t.WP2 > 0;
      const int Nt = pos ? 32 * t.WP1 * t.SPT : 0;
      if (tc ? (t.Rm < 1 || t.Rm > q.M) : (!pos || Nt < 32 || Nt > 128 || !tile_ok(t, q.L, q.p, q.M)))
        return fail(EDAA_ERR_ARG, "tile: launch shape outside the compiled register tiles or shared memory");
    }
  }
  edaa_ctx* c = new edaa_ctx();
  c->cfg = conf;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaGetDevice");
  }
  e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "device attribute");
  }
  c->stream = (cudaStream_t)stream;
  if (c->stream == nullptr || c->stream == cudaStreamLegacy) {
    e = cudaStreamCreate(&c->stream);  // blocking: ordered with the legacy stream
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "stream create");
    }
    c->own_stream = true;
  }
  memset(&c->hb, 0, sizeof(Batch));
  c->hb.n_cubes = n_cubes;
  c->hb.K1 = conf.K1;
  c->hb.K2 = conf.K2;
  c->hb.coh_mode = conf.coherence;
  c->hb.timeout_ns = (long long)(conf.barrier_timeout_ms * 1e6);
  c->hb.record_loss = conf.record_loss ? 1 : 0;
  c->hb.hist_cap = conf.record_loss ? std::max(conf.T, 1) : 0;
  for (int i = 0; i < n_cubes; ++i) {
    CubeHost h{};
    const edaa_cube& q = cubes[i];
    h.L = q.L; h.N = q.N; h.p = q.p; h.M = q.M;
    h.Ls = padded_ld(q.L);
    h.Lr = round_up(q.L, 4);
    h.Mp = q.M * q.p;
    h.hist_cap = c->hb.hist_cap;
    h.seeds.assign(q.seeds, q.seeds + q.M);
    h.gammas.assign(q.gammas, q.gammas + q.M);
    h.tile = default_tile(q.L, q.p, q.M);
    h.tile_fixed = conf.tile[0] != 0;  // validated above
    if (h.tile_fixed) h.tile = TileCfg{conf.tile[0], conf.tile[1], conf.tile[2], conf.tile[3]};
    h.tc_rm_fixed = conf.tile[0];
    // tensor cores only where the ensemble makes the contractions dense (M p >= 64)
    if (conf.precision != EDAA_FP32 && h.Mp >= 64) {
      h.tc = conf.precision == EDAA_BF16 ? 2 : (conf.precision == EDAA_TF32X3 ? 3 : 1);
      h.esz = h.tc == 2 ? 2 : 4;
      // bands per pixel row of the compute-type X (BF16: whole 64-band chunks,
      // at least two, as contraction 2 reads 128 bands per MMA)
      h.kp = h.tc == 2 ? 64 * tc_nkx(q.L) : round_up(q.L + 1, 128 / h.esz);
      h.Npad = round_up(q.N, 8);
      tc_tile(h);
    }
    memset(&h.dev, 0, sizeof(CubeDev));
    c->cubes.push_back(h);
  }
  // shared memory and occupancy: the largest need over cubes and candidates
  size_t smem = 0;
  for (auto& h : c->cubes) {
    smem = std::max(smem, pass_item_smem(h));
    smem = std::max(smem, (size_t)merge_smem(h.L, h.p, 256).total * 8);  // any band chunk, up to 256 partials
    if (conf.autotune && !h.tc)
      for (const auto& t : tile_candidates(h.L, h.p, h.M)) smem = std::max(smem, tile_smem(t, h.L, h.p));
  }
  smem = std::max(smem, (size_t)32 * 1024);
  c->smem = smem;
  // every tensor-core pass lays out its ring in this many bytes (narrower run
  // groups, e.g. the autotuner's candidates, take more stages, never more room)
  c->hb.smem_bytes = (unsigned)smem;
  auto bail = [&](edaa_status st) {
    edaa_destroy(c);
    return st;
  };
  e = set_program_smem(smem);
  if (e != cudaSuccess) return bail(cuda_fail(e, "set shared memory"));
  int bps = 0;
  e = program_occupancy(&bps, smem);
  if (e != cudaSuccess) return bail(cuda_fail(e, "occupancy"));
  if (bps < 1) return bail(fail(EDAA_ERR_UNSUPPORTED, "kernel does not fit on an SM"));
  c->blocks_per_sm = bps;
  plan(c);
  const int Gcap = c->sm_count * c->blocks_per_sm;
  for (auto& h : c->cubes) {
    const int ntiles_min = (h.N + 31) / 32;
    const int Pg_cap = std::max(1, std::min(Gcap, ntiles_min));
    h.arena_bytes = arena_layout(h, Pg_cap, false);
    e = dev_malloc(&h.arena, h.arena_bytes);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    e = cudaMemsetAsync(h.arena, 0, h.arena_bytes, c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "memset"));
    arena_layout(h, Pg_cap, true);
    if (h.tc) {
      edaa_status st = make_tmaps(c, h);
      if (st != EDAA_OK) return bail(st);
    }
  }
  e = dev_malloc((void**)&c->d_batch, sizeof(Batch));
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  e = dev_malloc((void**)&c->d_status, 64);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  c->d_bar = (unsigned*)(c->d_status + 4);
  c->hb.status = c->d_status;
  c->hb.bar = c->d_bar;
  c->hb.trace_start = c->hb.trace_end = nullptr;
  if (conf.trace) {
    e = dev_malloc((void**)&c->d_trace, (size_t)6 * kTraceCap * 8);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    c->hb.trace_start = c->d_trace;
    c->hb.trace_end = c->d_trace + 3 * kTraceCap;
  }
  for (size_t i = 0; i < c->cubes.size(); ++i) {
    CubeHost& h = c->cubes[i];
    e = cudaMemcpyAsync((void*)h.dev.seeds, h.seeds.data(), h.M * 8, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "copy seeds"));
    e = cudaMemcpyAsync((void*)h.dev.gammas, h.gammas.data(), h.M * 8, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "copy gammas"));
    edaa_status st = upload_x(c, h, cubes[i].X);
    if (st != EDAA_OK) return bail(st);
  }
  edaa_status st = push_batch(c);
  if (st != EDAA_OK) return bail(st);
  if (conf.autotune) {
    st = autotune(c);
    if (st != EDAA_OK) return bail(st);
  }
  st = run_init(c);
  if (st != EDAA_OK) return bail(st);
  *out = c;
  return EDAA_OK;
}

edaa_status edaa_reset(edaa_ctx* c, int cube, const float* X) {
  NvtxRange nvtx_range("edaa_reset");
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  edaa_status st = check_status(c);
  if (st != EDAA_OK) return st;
  if (X) {
    if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
    st = upload_x(c, c->cubes[cube], X);
    if (st != EDAA_OK) return st;
  } else if (cube < -1 || cube >= (int)c->cubes.size()) {
    return fail(EDAA_ERR_ARG, "cube index out of range");
  }
  return run_init(c);
}

edaa_status edaa_step(edaa_ctx* c, int n_outer) {
  NvtxRange nvtx_range("edaa_step");
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  if (n_outer < 0) return fail(EDAA_ERR_ARG, "n_outer must be >= 0");
  edaa_status st = check_status(c);
  if (st != EDAA_OK) return st;
  st = enqueue(c, MODE_OUTER, n_outer, nullptr);
  if (st == EDAA_OK) c->outer_done += n_outer;
  return st;
}

edaa_status edaa_solve(edaa_ctx* c) {
  NvtxRange nvtx_range("edaa_solve");
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  edaa_status st = check_status(c);
  if (st != EDAA_OK) return st;
  const int n = std::max(0, c->cfg.T - c->outer_done);
  int launches = 0;
  // graph: [outer iterations ; fit] captured once per n and replayed
  if (c->graphs_ok && c->g_solve_n != n) {
    if (c->g_solve) {
      cudaGraphExecDestroy(c->g_solve);
      c->g_solve = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      int l = 0;
      edaa_status s1 = enqueue(c, MODE_OUTER, n, &l);
      edaa_status s2 = (s1 == EDAA_OK) ? enqueue(c, MODE_FIT, 0, &l) : s1;
      e = cudaStreamEndCapture(c->stream, &g);
      if (e == cudaSuccess && s2 == EDAA_OK) e = cudaGraphInstantiate(&c->g_solve, g, 0);
      else if (e == cudaSuccess) e = cudaErrorUnknown;
      if (g) cudaGraphDestroy(g);
      if (e == cudaSuccess) {
        c->g_solve_n = n;
        c->launches_last_solve = l;
      }
    }
    if (e != cudaSuccess) {
      // reported, not fatal: this and later solves launch directly
      // (edaa_describe's graph state is -1 and edaa_last_error says why)
      g_err = std::string("CUDA-graph capture of the solve failed (solves launch directly): ") +
              cudaGetErrorString(e);
      cudaGetLastError();
      c->graphs_ok = false;
      c->g_solve = nullptr;
    }
  }
  if (c->graphs_ok && c->g_solve) {
    CK(cudaGraphLaunch(c->g_solve, c->stream), "graph launch");
    c->graph_state = 1;
  } else {
    c->graph_state = -1;
    st = enqueue(c, MODE_OUTER, n, &launches);
    if (st == EDAA_OK) st = enqueue(c, MODE_FIT, 0, &launches);
    if (st != EDAA_OK) return st;
    c->launches_last_solve = launches;
  }
  c->outer_done += n;
  return EDAA_OK;
}

edaa_status edaa_sync(edaa_ctx* c) {
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  edaa_status st = check_status(c);
  if (st != EDAA_OK) return st;
  return sync_status(c);
}

edaa_status edaa_select(edaa_ctx* c, int cube, int* best, double* fit, double* mu) {
  NvtxRange nvtx_range("edaa_select");
  if (!c || !best) return fail(EDAA_ERR_ARG, "ctx and best are required");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  edaa_status st = edaa_sync(c);
  if (st != EDAA_OK) return st;
  CubeHost& h = c->cubes[cube];
  std::vector<double> f(h.M), m(h.M);
  CK(cudaMemcpy(f.data(), c->cfg.fit_norm ? h.dev.fitmax : h.dev.fit, h.M * 8, cudaMemcpyDeviceToHost), "read fit");
  CK(cudaMemcpy(m.data(), h.dev.mu, h.M * 8, cudaMemcpyDeviceToHost), "read mu");
  if (fit) memcpy(fit, f.data(), h.M * 8);
  if (mu) memcpy(mu, m.data(), h.M * 8);
  *best = edaa_select_rule(f.data(), m.data(), h.M, c->cfg.fit_ratio);
  if (*best < 0) return fail(EDAA_ERR_NONFINITE, "no run has a finite fit");
  return EDAA_OK;
}

edaa_status edaa_get(edaa_ctx* c, int cube, int run, float* E, float* A, float* B) {
  NvtxRange nvtx_range("edaa_get");
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  CubeHost& h = c->cubes[cube];
  if (run < 0 || run >= h.M) return fail(EDAA_ERR_ARG, "run index out of range");
  edaa_status st = check_status(c);
  if (st != EDAA_OK) return st;
  // outputs may be host memory: gather into device scratch, then copy
  cudaPointerAttributes pa;
  auto is_dev = [&](const void* p) {
    if (!p) return true;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
  };
  const bool dE = is_dev(E), dA = is_dev(A), dB = is_dev(B);
  if (dE && dA && dB) {
    CK(launch_gather(h.dev, run, E, A, B, c->stream), "gather");
    return EDAA_OK;
  }
  const size_t nE = (size_t)h.L * h.p, nA = (size_t)h.N * h.p;
  float* tmp = nullptr;
  CK(dev_malloc_async((void**)&tmp, (nE + 2 * nA) * 4, c->stream), "scratch");
  float* tE = E ? (dE ? E : tmp) : nullptr;
  float* tA = A ? (dA ? A : tmp + nE) : nullptr;
  float* tB = B ? (dB ? B : tmp + nE + nA) : nullptr;
  CK(launch_gather(h.dev, run, tE, tA, tB, c->stream), "gather");
  if (E && !dE) CK(cudaMemcpyAsync(E, tE, nE * 4, cudaMemcpyDeviceToHost, c->stream), "copy E");
  if (A && !dA) CK(cudaMemcpyAsync(A, tA, nA * 4, cudaMemcpyDeviceToHost, c->stream), "copy A");
  if (B && !dB) CK(cudaMemcpyAsync(B, tB, nA * 4, cudaMemcpyDeviceToHost, c->stream), "copy B");
  CK(cudaFreeAsync(tmp, c->stream), "free scratch");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  return EDAA_OK;
}

edaa_status edaa_grad(edaa_ctx* c, int cube, int run, float* gA, float* gB) {
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  CubeHost& h = c->cubes[cube];
  if (run < 0 || run >= h.M) return fail(EDAA_ERR_ARG, "run index out of range");
  edaa_status st = check_status(c);
  if (st != EDAA_OK) return st;
  const size_t n = (size_t)h.N * h.p;
  float* tmp = nullptr;
  CK(dev_malloc_async((void**)&tmp, 2 * n * 4, c->stream), "scratch");
  const CubeDev* dcube = reinterpret_cast<const CubeDev*>(reinterpret_cast<const char*>(c->d_batch) +
                                                          offsetof(Batch, c) + (size_t)cube * sizeof(CubeDev));
  CK(launch_grad(dcube, h.dev, run, gA ? tmp : nullptr, gB ? tmp + n : nullptr, c->stream), "grad");
  if (gA) CK(cudaMemcpyAsync(gA, tmp, n * 4, cudaMemcpyDefault, c->stream), "copy gA");
  if (gB) CK(cudaMemcpyAsync(gB, tmp + n, n * 4, cudaMemcpyDefault, c->stream), "copy gB");
  CK(cudaFreeAsync(tmp, c->stream), "free scratch");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  return EDAA_OK;
}

edaa_status edaa_loss(edaa_ctx* c, int cube, double* loss) {
  NvtxRange nvtx_range("edaa_loss");
  if (!c || !loss) return fail(EDAA_ERR_ARG, "ctx and loss are required");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  edaa_status st = check_status(c);
  if (st != EDAA_OK) return st;
  st = enqueue(c, MODE_FIT, 0, nullptr);
  if (st != EDAA_OK) return st;
  st = sync_status(c);
  if (st != EDAA_OK) return st;
  CubeHost& h = c->cubes[cube];
  CK(cudaMemcpy(loss, h.dev.loss2, h.M * 8, cudaMemcpyDeviceToHost), "read loss");
  return EDAA_OK;
}

edaa_status edaa_loss_history(edaa_ctx* c, int cube, int cap, double* hist, int* n) {
  if (!c || !n) return fail(EDAA_ERR_ARG, "ctx and n are required");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  if (!c->hb.record_loss) return fail(EDAA_ERR_STATE, "the loss log is off (config.record_loss = 0)");
  edaa_status st = edaa_sync(c);
  if (st != EDAA_OK) return st;
  CubeHost& h = c->cubes[cube];
  const int rows = std::min(c->outer_done, h.hist_cap);
  *n = rows;
  const int k = std::min(rows, std::max(cap, 0));
  if (hist && k > 0)
    CK(cudaMemcpy(hist, h.dev.loss_hist, (size_t)k * h.M * 8, cudaMemcpyDeviceToHost), "read loss log");
  return EDAA_OK;
}

edaa_status edaa_checkpoint(edaa_ctx* c, void* buf, size_t cap, size_t* bytes) {
  if (!c || !bytes) return fail(EDAA_ERR_ARG, "ctx and bytes are required");
  edaa_status st = edaa_sync(c);
  if (st != EDAA_OK) return st;
  size_t total = sizeof(CkptHeader);
  for (auto& h : c->cubes) {
    total += sizeof(CkptCube) + (size_t)(h.L + 1) * 8;
    for (auto& r : state_regions(h)) total += r.bytes;
  }
  *bytes = total;
  if (!buf) return EDAA_OK;
  if (cap < total) return fail(EDAA_ERR_ARG, "checkpoint buffer too small (query the size with buf = NULL)");
  char* o = (char*)buf;
  CkptHeader hd{};
  memcpy(hd.magic, "EDAACKPT", 8);
  hd.version = 1;
  hd.n_cubes = (int)c->cubes.size();
  hd.outer_done = c->outer_done;
  hd.record_loss = c->hb.record_loss;
  hd.hist_cap = c->hb.hist_cap;
  hd.payload = total - sizeof(CkptHeader);
  memcpy(o, &hd, sizeof hd);
  o += sizeof hd;
  for (auto& h : c->cubes) {
    const CkptCube cc{h.L, h.N, h.p, h.M, h.tc, h.esz, h.kp, 0};
    memcpy(o, &cc, sizeof cc);
    o += sizeof cc;
    CK(cudaMemcpy(o, h.dev.sx, (size_t)(h.L + 1) * 8, cudaMemcpyDeviceToHost), "checkpoint");
    o += (size_t)(h.L + 1) * 8;
    for (auto& r : state_regions(h)) {
      CK(cudaMemcpy(o, r.ptr, r.bytes, cudaMemcpyDeviceToHost), "checkpoint");
      o += r.bytes;
    }
  }
  return EDAA_OK;
}

edaa_status edaa_restore(edaa_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return fail(EDAA_ERR_ARG, "ctx and buf are required");
  edaa_status st = edaa_sync(c);
  if (st != EDAA_OK) return st;
  const char* o = (const char*)buf;
  CkptHeader hd;
  if (bytes < sizeof hd) return fail(EDAA_ERR_ARG, "not a checkpoint (too short)");
  memcpy(&hd, o, sizeof hd);
  if (memcmp(hd.magic, "EDAACKPT", 8) != 0 || hd.version != 1) return fail(EDAA_ERR_ARG, "not a checkpoint");
  if (hd.payload + sizeof hd != bytes) return fail(EDAA_ERR_ARG, "checkpoint size does not match its header");
  if (hd.n_cubes != (int)c->cubes.size() || hd.record_loss != c->hb.record_loss || hd.hist_cap != c->hb.hist_cap)
    return fail(EDAA_ERR_ARG, "checkpoint taken on other cubes or another loss-log setting");
  o += sizeof hd;
  // check every cube before writing anything
  const char* q = o;
  for (auto& h : c->cubes) {
    CkptCube cc;
    memcpy(&cc, q, sizeof cc);
    if (cc.L != h.L || cc.N != h.N || cc.p != h.p || cc.M != h.M || cc.tc != h.tc || cc.esz != h.esz || cc.kp != h.kp)
      return fail(EDAA_ERR_ARG, "checkpoint taken on cubes of another shape or precision");
    q += sizeof cc;
    std::vector<double> sx(h.L + 1);
    CK(cudaMemcpy(sx.data(), h.dev.sx, sx.size() * 8, cudaMemcpyDeviceToHost), "restore");
    if (memcmp(sx.data(), q, sx.size() * 8) != 0)
      return fail(EDAA_ERR_ARG, "checkpoint taken on other data X (its band sums differ)");
    q += sx.size() * 8;
    for (auto& r : state_regions(h)) q += r.bytes;
  }
  for (auto& h : c->cubes) {
    o += sizeof(CkptCube) + (size_t)(h.L + 1) * 8;
    for (auto& r : state_regions(h)) {
      CK(cudaMemcpyAsync(r.ptr, o, r.bytes, cudaMemcpyHostToDevice, c->stream), "restore");
      o += r.bytes;
    }
  }
  CK(cudaStreamSynchronize(c->stream), "restore");
  c->outer_done = hd.outer_done;
  return EDAA_OK;
}

edaa_status edaa_step_sizes(edaa_ctx* c, int cube, double* eta1, double* eta2) {
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  edaa_status st = edaa_sync(c);
  if (st != EDAA_OK) return st;
  CubeHost& h = c->cubes[cube];
  if (eta1) CK(cudaMemcpy(eta1, h.dev.eta1d, h.M * 8, cudaMemcpyDeviceToHost), "read eta1");
  if (eta2) CK(cudaMemcpy(eta2, h.dev.eta2d, h.M * 8, cudaMemcpyDeviceToHost), "read eta2");
  return EDAA_OK;
}

int edaa_outer_done(const edaa_ctx* c) { return c ? c->outer_done : -1; }

edaa_status edaa_describe(const edaa_ctx* c, int cube, int* runs_per_group, int* pixel_tile, int* ctas_per_group,
                          int* grid, int* launches_per_solve, int* graph_state) {
  if (!c) return fail(EDAA_ERR_ARG, "ctx is NULL");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  const CubeHost& h = c->cubes[cube];
  if (runs_per_group) *runs_per_group = h.tile.Rm;
  if (pixel_tile) *pixel_tile = h.Nt;
  if (ctas_per_group) *ctas_per_group = h.Pg;
  if (grid) *grid = c->grid;
  if (launches_per_solve) *launches_per_solve = c->launches_last_solve;
  if (graph_state) *graph_state = c->graph_state;
  return EDAA_OK;
}

edaa_status edaa_describe_tile(const edaa_ctx* c, int cube, int tile[4]) {
  if (!c || !tile) return fail(EDAA_ERR_ARG, "ctx or tile is NULL");
  if (cube < 0 || cube >= (int)c->cubes.size()) return fail(EDAA_ERR_ARG, "cube index out of range");
  const TileCfg& t = c->cubes[cube].tile;
  tile[0] = t.Rm;
  tile[1] = t.WP1;
  tile[2] = t.SPT;
  tile[3] = t.WP2;
  return EDAA_OK;
}

edaa_status edaa_trace_read(edaa_ctx* c, int which, int cap, int* n, int* phase, double* start_us, double* dur_us) {
  if (!c || !n) return fail(EDAA_ERR_ARG, "ctx or n is NULL");
  if (which < 0 || which > 2) return fail(EDAA_ERR_ARG, "which must be 0, 1 or 2");
  if (!c->d_trace) return fail(EDAA_ERR_STATE, "tracing is off (config.trace = 0)");
  const int m = c->trace_n[which];
  std::vector<unsigned long long> t0(std::max(m, 1)), t1(std::max(m, 1));
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  if (m > 0) {
    CK(cudaMemcpy(t0.data(), c->d_trace + (size_t)which * kTraceCap, (size_t)m * 8, cudaMemcpyDeviceToHost), "read trace");
    CK(cudaMemcpy(t1.data(), c->d_trace + (size_t)(3 + which) * kTraceCap, (size_t)m * 8, cudaMemcpyDeviceToHost),
       "read trace");
  }
  const unsigned long long base = m > 0 ? t0[0] : 0;
  for (int i = 0; i < m && i < cap; ++i) {
    if (phase) phase[i] = program_phase_id(which, i, c->cfg.K2, c->hb.record_loss);
    if (start_us) start_us[i] = ((double)t0[i] - (double)base) * 1e-3;
    if (dur_us) dur_us[i] = ((double)t1[i] - (double)t0[i]) * 1e-3;
  }
  *n = m;
  return EDAA_OK;
}

void edaa_destroy(edaa_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->g_solve) cudaGraphExecDestroy(c->g_solve);
  for (auto& h : c->cubes)
    if (h.arena) cudaFree(h.arena);
  if (c->d_batch) cudaFree(c->d_batch);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_trace) cudaFree(c->d_trace);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

edaa_status edaa_measure_fma_peak(double* tflops, void* stream) {
  if (!tflops) return fail(EDAA_ERR_ARG, "tflops is NULL");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = sms * 8, iters = 1 << 16;
  float* out = nullptr;
  CK(cudaMalloc(&out, (size_t)blocks * 256 * sizeof(float)), "cudaMalloc");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 0.0;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_fma_peak(out, blocks, iters, s);  // warm-up
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_fma_peak(out, blocks, iters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f) best = std::max(best, fma_peak_flops_per_launch(blocks, iters) / (ms * 1e-3) / 1e12);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "FMA probe");
  *tflops = best;
  return EDAA_OK;
}

void edaa_debug_fail_alloc(int k) { g_fail_alloc.store(k < 0 ? -1 : k); }

edaa_status edaa_selftest_barrier(int grid, int extra, double timeout_ms, void* stream) {
  if (grid < 1 || grid > 4096 || extra < 0) return fail(EDAA_ERR_ARG, "grid must be 1..4096, extra >= 0");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  if (grid > sms) return fail(EDAA_ERR_ARG, "grid must not exceed the SM count (co-residency)");
  cudaStream_t s = (cudaStream_t)stream;
  int* buf = nullptr;
  CK(cudaMalloc(&buf, 64), "cudaMalloc");
  cudaError_t e = cudaMemsetAsync(buf, 0, 64, s);
  if (e == cudaSuccess)
    e = launch_barrier_test((unsigned*)(buf + 4), buf, grid, grid + extra, (long long)(timeout_ms * 1e6), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, buf, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "barrier self-test");
  if (st & kStatTimeout) return fail(EDAA_ERR_TIMEOUT, "barrier timed out as expected");
  return EDAA_OK;
}

}  // extern "C"
