// C ABI of libtpd.so (declared in include/tpd.h): argument checks, the plan
// cache, workspace layout and the launch sequence of each call.  Host code
// only; the kernels are behind the launchers of tpd_launch.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "tpd.h"
#include "tpd_launch.h"
#include "tpd_planner.h"

namespace tpd {
namespace {

std::mutex g_plan_mu;
std::map<std::tuple<int, int, int, int, int>, Plan> g_plans;

int resolve_precision(int dtype, int precision) {
  if (precision == TPD_PREC_DEFAULT) return dtype == TPD_C128 ? TPD_PREC_FIXED : TPD_PREC_PLAIN;
  return precision;
}

int arith_of(int dtype, int prec) {
  if (dtype == TPD_C128) return prec == TPD_PREC_FIXED ? kArithFixed : kArithF64;
  if (prec == TPD_PREC_FIXED) return kArithF32Fixed;
  return prec == TPD_PREC_COMPENSATED ? kArithF32C : kArithF32;
}

tpd_status check_options(int dtype, const tpd_options* opt, int* prec) {
  if (dtype != TPD_C128 && dtype != TPD_C64) return TPD_ERR_INVALID_ARG;
  const int p = resolve_precision(dtype, opt ? opt->precision : 0);
  if (p < TPD_PREC_PLAIN || p > TPD_PREC_FIXED) return TPD_ERR_INVALID_ARG;
  if (p == TPD_PREC_COMPENSATED && dtype != TPD_C64) return TPD_ERR_UNSUPPORTED;
  if (opt && opt->tile_bits != 0 && (opt->tile_bits < kMinTileBits || opt->tile_bits > kMaxTileBits))
    return TPD_ERR_INVALID_ARG;
  if (opt && (opt->max_levels < 0 || opt->max_levels > kMaxLevels)) return TPD_ERR_INVALID_ARG;
  if (opt && (opt->variant < 0 || opt->variant > 4)) return TPD_ERR_INVALID_ARG;
  *prec = p;
  return TPD_OK;
}

tpd_status check_common(int n, int dtype, const tpd_options* opt, int* prec) {
  if (n < 1 || n > kMaxQubits) return TPD_ERR_INVALID_ARG;
  return check_options(dtype, opt, prec);
}

// Tuned defaults (tpd_tune_set): (n, dtype, precision) -> tile_bits, max_levels, variant.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> g_tuned;

// The caller's options, with the tuned defaults filled in when it left all
// three tuning fields at 0.
tpd_options effective_options(int n, int dtype, int prec, const tpd_options* opt) {
  tpd_options e;
  if (opt) e = *opt;
  else std::memset(&e, 0, sizeof(e));
  if (e.tile_bits == 0 && e.max_levels == 0 && e.variant == 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(n, dtype, prec));
    if (it != g_tuned.end()) {
      e.tile_bits = std::get<0>(it->second);
      e.max_levels = std::get<1>(it->second);
      e.variant = std::get<2>(it->second);
    }
  }
  return e;
}

// Cached plan for (n, dtype, precision, tuning options); nullptr if impossible.
const Plan* get_plan(int n, int dtype, int prec, const tpd_options* opt) {
  const int tb = opt ? opt->tile_bits : 0, ml = opt ? opt->max_levels : 0;
  const auto key = std::make_tuple(n, dtype, prec, tb, ml);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find(key);
  if (it != g_plans.end()) return &it->second;
  Plan p;
  std::string err;
  if (!build_plan(n, dtype, prec, tb, ml, &p, &err)) return nullptr;
  return &g_plans.emplace(key, p).first->second;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }


// Workspace of one matrix's plan:
//   zero-skip flags: one byte per tile of every pass after the first (skip only)
//   binary points:   one int per tile of every pass but the last (fixed point only)
struct Layout {
  size_t flags_off[kMaxQubits];
  size_t q_off[kMaxQubits];
  size_t flags_bytes, q_bytes, total;
};

Layout layout_of(const Plan& p, int arith, int skip) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  size_t off = 0;
  if (skip)
    for (int i = 1; i < p.npass; ++i) { L.flags_off[i] = off; off += (size_t)p.pass[i].ntiles; }
  L.flags_bytes = align256(off);
  off = L.flags_bytes;
  if (arith == kArithFixed)
    for (int i = 0; i + 1 < p.npass; ++i) { L.q_off[i] = off; off += (size_t)p.pass[i].ntiles * sizeof(int); }
  L.q_bytes = align256(off) - L.flags_bytes;
  L.total = L.flags_bytes + L.q_bytes;
  return L;
}

// Composition scale = m * 2^e; exact power of two when m == 1/2 in frexp form.
void split_scale(double scale, int* pow2, double* residual) {
  int e = 0;
  const double fr = std::frexp(scale, &e);
  if (fr == 0.5) { *pow2 = e - 1; *residual = 1.0; }
  else { *pow2 = 0; *residual = scale; }
}

void pass_scaling(bool dec, int arith, const PassDesc& pd, bool last, int spow, double sres, double scale,
                  PassArgs* a) {
  if (arith == kArithFixed || arith == kArithF32Fixed) {
    // the kernel folds the 1/2 of Eq. 4 into its binary point; only the
    // composition's scale is applied here, on the last pass
    a->out_pow2 = (!dec && last) ? spow : 0;
    a->out_mul = (!dec && last) ? sres : 1.0;
  } else if (dec) {
    a->out_pow2 = -pd.K;                            // the 1/2 of Eq. 4, once per fused level
    a->out_mul = std::ldexp(1.0, -pd.K);
  } else {
    a->out_pow2 = last ? spow : 0;
    a->out_mul = last ? scale : 1.0;
  }
}

// SM count of the current device (cached per device)
int sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 132;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 132;
    cache[dev] = v;
  }
  return cache[dev];
}

// profiling hook: event k recorded before pass k (k = 0) / after pass k-1
void record_event(const tpd_options* opt, int k, cudaStream_t s) {
  if (opt && opt->pass_events && k < opt->num_events && opt->pass_events[k])
    cudaEventRecord(static_cast<cudaEvent_t>(opt->pass_events[k]), s);
}

// L2 chunking of a single matrix's first passes: F passes (0 = none) and the
// global bits fixed per chunk (ascending).  The union U of the first F
// passes' tile bits leaves 2n - |U| bits outside every one of their tiles;
// all but the lowest g of them are fixed per chunk, g chosen so a chunk
// (2^(|U| + g) elements) fits the budget.  F is the most passes whose chunk
// still fits; chunking pays only when F >= 2.
struct L2Chunks {
  int F = 0;
  std::vector<int> fixed;
};

L2Chunks l2_chunks(const Plan& plan, const tpd_options* opt, bool off) {
  L2Chunks r;
  const int mb = opt ? opt->l2_chunk_mb : 0;
  if (off || mb <= 0 || plan.npass < 2) return r;
  const double budget = mb * 1048576.0;
  const int nb = 2 * plan.n;
  unsigned long long uni = 0;
  int best_F = 0;
  unsigned long long best_uni = 0;
  for (int F = 1; F < plan.npass; ++F) {
    const PassDesc& pd = plan.pass[F - 1];
    for (int i = 0; i < pd.D; ++i) uni |= 1ull << pd.gbit[i];
    const int u = __builtin_popcountll(uni);
    if (u >= nb || std::ldexp((double)plan.elem_bytes, u) > budget) break;
    best_F = F;
    best_uni = uni;
  }
  if (best_F < 2) return r;
  const int u = __builtin_popcountll(best_uni);
  int g = 0;
  while (u + g + 1 <= nb && std::ldexp((double)plan.elem_bytes, u + g + 1) <= budget) ++g;
  int skipped = 0;
  for (int b = 0; b < nb; ++b) {
    if ((best_uni >> b) & 1ull) continue;
    if (skipped < g) { ++skipped; continue; }      // the lowest g outside bits stay free in a chunk
    r.fixed.push_back(b);
  }
  if (r.fixed.empty()) return r;
  r.F = best_F;
  return r;
}

tpd_status run_single(bool dec, int arith, void* mat, const Plan& plan, int skip, double scale, void* ws,
                      cudaStream_t s, const tpd_options* opt, const uint8_t* const* need = nullptr) {
  record_event(opt, 0, s);
  if (plan.npass == 0) {
    SmallArgs a;
    std::memset(&a, 0, sizeof(a));
    a.mat = mat; a.n = plan.n; a.skip_zero = skip;
    a.scale_mode = dec ? 0 : (scale == 1.0 ? 0 : 1);
    if (launch_small(arith, dec, a, 1, plan.n, s) != cudaSuccess) return TPD_ERR_CUDA;
    record_event(opt, 1, s);
    return TPD_OK;
  }
  const Layout lay = layout_of(plan, arith, skip);
  char* w = static_cast<char*>(ws);
  if (skip && lay.flags_bytes && cudaMemsetAsync(w, 0, lay.flags_bytes, s) != cudaSuccess) return TPD_ERR_CUDA;
  // with skipping, tiles a pass never visits keep the "zero tile" fill
  if (skip && lay.q_bytes && cudaMemsetAsync(w + lay.flags_bytes, kQFillByte, lay.q_bytes, s) != cudaSuccess)
    return TPD_ERR_CUDA;
  int spow = 0;
  double sres = 1.0;
  if (!dec) split_scale(scale, &spow, &sres);
  const int variant = opt ? opt->variant : 0;
  auto pass_args = [&](int p) {
    const PassDesc& pd = plan.pass[p];
    const bool last = p + 1 == plan.npass;
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.mat = mat;
    a.skip_zero = skip;
    if (skip && p > 0) a.flags_in = reinterpret_cast<uint8_t*>(w + lay.flags_off[p]);
    if (skip && !last) a.flags_out = reinterpret_cast<uint8_t*>(w + lay.flags_off[p + 1]);
    if (need) a.need = need[p];
    if (arith == kArithFixed) {
      if (p > 0) a.q_in = reinterpret_cast<const int*>(w + lay.q_off[p - 1]);
      if (!last) a.q_out = reinterpret_cast<int*>(w + lay.q_off[p]);
    }
    pass_scaling(dec, arith, pd, last, spow, sres, scale, &a);
    return a;
  };
  auto tuned_desc = [&](int p) {
    PassDesc tuned = plan.pass[p];            // occupancy override (variants 3 and 4)
    if (tuned.D <= 12 && (variant == 3 || variant == 4)) tuned.min_blocks = variant == 3 ? 2 : 3;
    return tuned;
  };
  // L2 chunking: the first F passes run chunk by chunk, each chunk (the
  // elements that agree on the global bits outside all F passes' tiles) small
  // enough to stay in L2 from one pass to the next.
  const L2Chunks ch = l2_chunks(plan, opt, skip || need || variant == 2);
  int p0 = 0;
  if (ch.F >= 2) {
    const int nfix = (int)ch.fixed.size();
    for (unsigned long long c = 0; c < (1ull << nfix); ++c)
      for (int p = 0; p < ch.F; ++p) {
        const PassDesc& pd = plan.pass[p];
        PassArgs a = pass_args(p);
        a.chunked = 1;
        a.chunk_or = 0;
        a.nfree = 0;
        for (int j = 0; j < pd.nrest; ++j) {
          int k = 0;
          while (k < nfix && ch.fixed[k] != pd.rest_gbit[j]) ++k;
          if (k < nfix) a.chunk_or |= ((c >> k) & 1ull) << j;
          else a.chunk_free[a.nfree++] = (int8_t)j;
        }
        if (launch_pass(arith, dec, tuned_desc(p), a, 1ll << a.nfree, s) != cudaSuccess) return TPD_ERR_CUDA;
      }
    for (int p = 0; p < ch.F; ++p) record_event(opt, p + 1, s);
    p0 = ch.F;
  }
  for (int p = p0; p < plan.npass; ++p) {
    const PassDesc& pd = plan.pass[p];
    const PassArgs a = pass_args(p);
    const bool pipe = arith == kArithFixed && !skip && !need && pd.D <= 12 && variant == 2;
    const PassDesc tuned = tuned_desc(p);
    cudaError_t e = pipe ? launch_pass_pipe_c128(dec, tuned, a, sm_count(), s)
                         : launch_pass(arith, dec, tuned, a, pd.ntiles, s);
    if (e != cudaSuccess) return TPD_ERR_CUDA;
    record_event(opt, p + 1, s);
  }
  return TPD_OK;
}

size_t single_ws(const Plan& plan, int arith, int skip) {
  return plan.npass > 1 ? layout_of(plan, arith, skip).total : 0;
}

tpd_status single(bool dec, void* mat, int n, int dtype, double scale, const tpd_options* opt_in, void* ws,
                  size_t ws_bytes, void* stream) {
  int prec = 0;
  tpd_status st = check_common(n, dtype, opt_in, &prec);
  if (st != TPD_OK) return st;
  const tpd_options eff = effective_options(n, dtype, prec, opt_in);
  const tpd_options* opt = &eff;
  if (mat == nullptr) return TPD_ERR_INVALID_ARG;
  const size_t align = dtype == TPD_C128 ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(mat) % align) return TPD_ERR_MISALIGNED;
  if (!dec && (!std::isfinite(scale) || scale == 0.0)) return TPD_ERR_INVALID_ARG;
  const Plan* plan = get_plan(n, dtype, prec, opt);
  if (!plan) return TPD_ERR_INVALID_ARG;
  if (!dec && plan->npass == 0 && scale != 1.0 && scale != std::ldexp(1.0, -n))
    return TPD_ERR_UNSUPPORTED;  // whole-matrix kernel: scale 1 or 2^-n
  const int skip = opt ? (opt->skip_zero != 0) : 0;
  const int arith = arith_of(dtype, prec);
  const size_t need = single_ws(*plan, arith, skip);
  if (need && (ws == nullptr || ws_bytes < need)) return TPD_ERR_WORKSPACE;
  if (ws && reinterpret_cast<uintptr_t>(ws) % 16) return TPD_ERR_MISALIGNED;
  return run_single(dec, arith, mat, *plan, skip, scale, ws, static_cast<cudaStream_t>(stream), opt);
}

// ------------------------------------------------------------------ partial decomposition
//
// Only the weights of a requested list of strings (Alg. 3: a quaternary
// subtree T of the strings of interest).  The passes run in place as usual,
// but a pass skips every tile that no requested weight depends on: the last
// pass needs the tiles holding a requested position; an earlier pass needs
// the tiles that share elements with a needed tile of the pass after it
// (tiles of consecutive passes share elements iff they agree on the global
// bits fixed in both).  Needed tiles are computed exactly as in the full
// decomposition, so the requested weights carry the same bits.

// workspace: RC positions of the requested strings | per pass, one byte per
// tile: needed | the plan's own workspace (binary points between passes)
struct PartialLayout {
  size_t need_off[kMaxQubits];
  size_t run_off, run_bytes, total;
};

PartialLayout partial_layout(const Plan& plan, int arith, size_t count) {
  PartialLayout L;
  std::memset(&L, 0, sizeof(L));
  size_t off = align256(count * sizeof(unsigned long long));
  for (int p = 0; p < plan.npass; ++p) { L.need_off[p] = off; off += align256((size_t)plan.pass[p].ntiles); }
  L.run_off = off;
  L.run_bytes = single_ws(plan, arith, 0);
  L.total = off + L.run_bytes;
  return L;
}

// base-4 string index (t_1 most significant: digit b from the right is the
// symbol of qubit n-b, on row bit r_b and column bit c_b) -> RC position
unsigned long long rc_of_string(unsigned long long sidx, int n) {
  unsigned long long r = 0, c = 0;
  for (int b = 0; b < n; ++b) {
    c |= ((sidx >> (2 * b)) & 1ull) << b;
    r |= ((sidx >> (2 * b + 1)) & 1ull) << b;
  }
  return (r << n) | c;
}

unsigned long long tile_base_of(const PassDesc& pd, unsigned long long t) {
  unsigned long long b = 0;
  for (int j = 0; j < pd.nrest; ++j)
    if ((t >> j) & 1ull) b |= 1ull << pd.rest_gbit[j];
  return b;
}
unsigned long long tile_of(const PassDesc& pd, unsigned long long pos) {
  unsigned long long t = 0;
  for (int j = 0; j < pd.nrest; ++j) t |= ((pos >> pd.rest_gbit[j]) & 1ull) << j;
  return t;
}
unsigned long long fixed_mask(const PassDesc& pd) {
  unsigned long long m = 0;
  for (int j = 0; j < pd.nrest; ++j) m |= 1ull << pd.rest_gbit[j];
  return m;
}

void partial_need(const Plan& plan, const std::vector<unsigned long long>& pos,
                  std::vector<std::vector<uint8_t>>* need) {
  const int P = plan.npass;
  need->assign(P, {});
  for (int p = 0; p < P; ++p) (*need)[p].assign((size_t)plan.pass[p].ntiles, 0);
  for (unsigned long long x : pos) (*need)[P - 1][tile_of(plan.pass[P - 1], x)] = 1;
  for (int q = P - 2; q >= 0; --q) {
    const PassDesc& a = plan.pass[q];
    const PassDesc& b = plan.pass[q + 1];
    const unsigned long long C = fixed_mask(a) & fixed_mask(b);
    std::vector<unsigned long long> keys;
    for (unsigned long long t = 0; t < (unsigned long long)b.ntiles; ++t)
      if ((*need)[q + 1][t]) keys.push_back(tile_base_of(b, t) & C);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    for (unsigned long long t = 0; t < (unsigned long long)a.ntiles; ++t)
      (*need)[q][t] = std::binary_search(keys.begin(), keys.end(), tile_base_of(a, t) & C) ? 1 : 0;
  }
}

tpd_status partial_setup(int n, int dtype, const tpd_options* opt_in, int* prec, int* arith, const Plan** plan,
                         tpd_options* eff) {
  tpd_status st = check_common(n, dtype, opt_in, prec);
  if (st != TPD_OK) return st;
  if (opt_in && opt_in->skip_zero) return TPD_ERR_UNSUPPORTED;
  *eff = effective_options(n, dtype, *prec, opt_in);
  *plan = get_plan(n, dtype, *prec, eff);
  if (!*plan) return TPD_ERR_INVALID_ARG;
  *arith = arith_of(dtype, *prec);
  return TPD_OK;
}

// ------------------------------------------------------------------ batched
constexpr int kBatchMaxQubits = kBatchMaxN;
static_assert(kBatchStatusTimeout == TPD_ERR_TIMEOUT && kBatchStatusBadSizes == TPD_ERR_INVALID_ARG,
              "device status codes are tpd_status values");
static_assert(sizeof(BatchParams) <= 32000, "kernel parameter space");

bool g_hold_batch_waits = false;   // test hook (tpd_test_hold_batch_waits)

// workspace: control words (status, work counter, per-matrix pass completion
// counters of the persistent kernel) | items[count] (matrix indices bucketed
// by qubit count, on the device) | per qubit count n (ascending), for the fixed point: binary
// points of hist[n] matrices for every pass but the last
size_t batched_q_bytes(const Plan& plan, int arith, int count_n) {
  if (arith != kArithFixed || plan.npass < 2) return 0;
  size_t b = 0;
  for (int i = 0; i + 1 < plan.npass; ++i) b += (size_t)plan.pass[i].ntiles * sizeof(int) * (size_t)count_n;
  return align256(b);
}
size_t batched_ctrl(const int* hist, const std::vector<const Plan*>& plans) {
  size_t words = kCtrlDone;
  for (int n = 1; n <= kBatchMaxQubits; ++n)
    if (hist[n] && plans[n]->npass > 1) words += (size_t)hist[n] * (plans[n]->npass - 1);
  return align256(words * sizeof(unsigned));
}
size_t batched_head(int count) { return align256((size_t)count * sizeof(int)); }

// Options a batched call plans qubit count n with: the caller's (or tuned)
// choices; for the one-launch form (variant 2) n >= 7 defaults to
// 2^12-element tiles, the persistent kernel's tile.
tpd_options batch_options(int n, int dtype, int prec, const tpd_options* opt) {
  tpd_options eff = effective_options(n, dtype, prec, opt);
  const int caller_variant = opt ? opt->variant : 0;
  if (caller_variant == 2 && n >= 7 && eff.tile_bits == 0) eff.tile_bits = 12;
  return eff;
}

// The persistent form applies when every matrix is either small (n <= 6: one
// work item, whole matrix in shared memory) or planned with 2^12-element
// tiles (256-thread CTAs) in at most kSegMaxPasses passes, and the work list
// fits the kernel's parameters.
bool persistent_fits(const int* hist, const std::vector<const Plan*>& plans) {
  int ndesc = 0;
  long long items = 1;
  for (int n = 1; n <= kBatchMaxQubits; ++n) {
    if (!hist[n]) continue;
    const Plan& p = *plans[n];
    if (n <= 6) { items += hist[n]; continue; }
    if (p.npass > kSegMaxPasses) return false;
    for (int i = 0; i < p.npass; ++i)
      if (p.pass[i].D != 12) return false;
    ndesc += p.npass;
    items += (long long)(hist[n] + (p.npass - 1) * 4096) * p.npass * p.pass[0].ntiles;   // lag <= 4096
  }
  return ndesc <= kBatchMaxDescs && items < 0x7fffffffll;
}

// Work list of the persistent kernel (see tpd_launch.h): bucketing, one
// pipelined segment per qubit count n >= 7 (largest first), then the small
// matrices (largest first).
tpd_status run_persistent(bool dec, int arith, void* const* ptrs_dev, const int* ns_dev, int count, const int* hist,
                          const std::vector<const Plan*>& plans, int scale_mode, unsigned* ctrl, int* items,
                          char* qbase0, size_t ctrl_bytes, cudaStream_t s) {
  static BatchParams bp;               // large: built under the lock, copied into the launch
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  std::memset(&bp, 0, sizeof(bp));
  bp.count = count;
  for (int n = 0; n <= kBatchMaxQubits; ++n) bp.hist[n] = hist[n];
  bp.scale_mode = dec ? 0 : scale_mode;
  bp.ptrs = ptrs_dev; bp.ns = ns_dev; bp.items = items; bp.ctrl = ctrl;
  int item_start[kBatchMaxQubits + 2] = {0};
  for (int n = 1; n <= kBatchMaxQubits + 1; ++n) item_start[n] = item_start[n - 1] + hist[n - 1];
  // per n (ascending, as the workspace lays them out): q area and done-counter base
  size_t qbase_n[kBatchMaxQubits + 1] = {0};
  int dbase_n[kBatchMaxQubits + 1] = {0};
  {
    size_t q = 0;
    int d = 0;
    for (int n = 1; n <= kBatchMaxQubits; ++n) {
      if (!hist[n]) continue;
      qbase_n[n] = q;
      dbase_n[n] = d;
      q += batched_q_bytes(*plans[n], arith, hist[n]);
      if (plans[n]->npass > 1) d += hist[n] * (plans[n]->npass - 1);
    }
  }
  // CTAs in flight: 2 per SM; a matrix's later pass trails its previous pass
  // by at least twice that many items, so the tiles it waits for are done
  const long long inflight = 2ll * sm_count();
  long long first = 1;
  int nseg = 0, ndesc = 0;
  for (int n = kBatchMaxQubits; n >= 7; --n) {
    if (!hist[n]) continue;
    const Plan& p = *plans[n];
    BatchSeg& sg = bp.seg[nseg++];
    sg.kind = kSegPipe; sg.n = n; sg.npass = p.npass; sg.desc = ndesc;
    sg.item_start = item_start[n]; sg.nmat = hist[n];
    sg.tiles = p.pass[0].ntiles;
    const long long per_round = (long long)p.npass * sg.tiles;
    long long lag = (2 * inflight + per_round - 1) / per_round;
    sg.lag = (int)(lag < 1 ? 1 : (lag > 4096 ? 4096 : lag));
    sg.done = dbase_n[n];
    sg.wait_extra = g_hold_batch_waits ? 1 : 0;
    sg.first = first;
    size_t qoff = qbase_n[n];
    for (int i = 0; i < p.npass; ++i) {
      const PassDesc& pd = p.pass[i];
      const bool last = i + 1 == p.npass;
      bp.desc[ndesc++] = pd;
      PassArgs& a = sg.args[i];
      if (arith == kArithFixed) {
        if (i > 0) {
          a.q_in = sg.args[i - 1].q_out;
          a.q_in_stride = p.pass[i - 1].ntiles;
        }
        if (!last) {
          a.q_out = reinterpret_cast<int*>(qbase0 + qoff);
          a.q_out_stride = pd.ntiles;
          qoff += (size_t)pd.ntiles * sizeof(int) * hist[n];
        }
      }
      const double scale = scale_mode ? std::ldexp(1.0, -n) : 1.0;
      pass_scaling(dec, arith, pd, last, scale_mode ? -n : 0, 1.0, scale, &a);
    }
    first += (long long)(hist[n] + (long long)(p.npass - 1) * sg.lag) * per_round;
  }
  for (int n = 6; n >= 1; --n) {
    if (!hist[n]) continue;
    BatchSeg& sg = bp.seg[nseg++];
    sg.kind = kSegSmall; sg.n = n; sg.npass = 0; sg.desc = -1;
    sg.item_start = item_start[n]; sg.nmat = hist[n];
    sg.first = first; sg.tiles = 1;
    first += hist[n];
  }
  bp.nseg = nseg;
  bp.total = first;
  if (cudaMemsetAsync(ctrl, 0, ctrl_bytes, s) != cudaSuccess) return TPD_ERR_CUDA;
  if (launch_batch(arith, dec, bp, nullptr, s) != cudaSuccess) return TPD_ERR_CUDA;
  return TPD_OK;
}

tpd_status batched(bool dec, void* const* ptrs_dev, const int* ns_dev, const int* ns, int count, int dtype,
                   int scale_mode, const tpd_options* opt, void* ws, size_t ws_bytes, void* stream) {
  int prec = 0;
  tpd_status st = check_options(dtype, opt, &prec);
  if (st != TPD_OK) return st;
  if (count < 0 || (count > 0 && (ptrs_dev == nullptr || ns_dev == nullptr || ns == nullptr)))
    return TPD_ERR_INVALID_ARG;
  if (scale_mode != 0 && scale_mode != 1) return TPD_ERR_INVALID_ARG;
  if (opt && opt->skip_zero) return TPD_ERR_UNSUPPORTED;
  if (count == 0) return TPD_OK;
  int hist[kBatchMaxQubits + 1] = {0};
  for (int i = 0; i < count; ++i) {
    if (ns[i] < 1 || ns[i] > kBatchMaxQubits) return TPD_ERR_INVALID_ARG;
    hist[ns[i]]++;
  }
  const int arith = arith_of(dtype, prec);
  std::vector<const Plan*> plans(kBatchMaxQubits + 1, nullptr);
  std::vector<int> variants(kBatchMaxQubits + 1, 0);
  size_t need = batched_head(count);
  for (int n = 1; n <= kBatchMaxQubits; ++n) {
    if (!hist[n]) continue;
    const tpd_options eff = batch_options(n, dtype, prec, opt);   // tuned per qubit count
    if (!(plans[n] = get_plan(n, dtype, prec, &eff))) return TPD_ERR_INVALID_ARG;
    variants[n] = eff.variant;
    need += batched_q_bytes(*plans[n], arith, hist[n]);
  }
  const size_t ctrl_bytes = batched_ctrl(hist, plans);
  need += ctrl_bytes;
  if (ws == nullptr || ws_bytes < need) return TPD_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 16) return TPD_ERR_MISALIGNED;
  unsigned* ctrl = static_cast<unsigned*>(ws);
  int* items = reinterpret_cast<int*>(static_cast<char*>(ws) + ctrl_bytes);
  char* qbase = reinterpret_cast<char*>(items) + batched_head(count);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int caller_variant = opt ? opt->variant : 0;
  if (caller_variant == 2 && persistent_fits(hist, plans))
    return run_persistent(dec, arith, ptrs_dev, ns_dev, count, hist, plans, scale_mode, ctrl, items, qbase,
                          ctrl_bytes, s);
  if (cudaMemsetAsync(ctrl, 0, ctrl_bytes, s) != cudaSuccess) return TPD_ERR_CUDA;   // status word: OK
  BucketHist bh;
  for (int n = 0; n <= kBatchMaxQubits; ++n) bh.h[n] = hist[n];
  if (launch_bucket(ns_dev, count, bh, items, ctrl + kCtrlStatus, s) != cudaSuccess) return TPD_ERR_CUDA;
  int start = 0;  // first bucket position of qubit count n: buckets are in increasing n
  for (int n = 1; n <= kBatchMaxQubits; ++n) {
    if (!hist[n]) continue;
    const Plan& plan = *plans[n];
    const int* its = items + start;
    if (plan.npass == 0) {
      SmallArgs a;
      std::memset(&a, 0, sizeof(a));
      a.ptrs = ptrs_dev; a.ns = ns_dev; a.items = its;
      a.scale_mode = dec ? 0 : scale_mode;
      if (launch_small(arith, dec, a, hist[n], n, s) != cudaSuccess) return TPD_ERR_CUDA;
    } else {
      size_t qoff = 0;
      const int* q_prev = nullptr;
      long long q_prev_stride = 0;
      for (int p = 0; p < plan.npass; ++p) {
        const PassDesc& pd = plan.pass[p];
        const bool last = p + 1 == plan.npass;
        PassArgs a;
        std::memset(&a, 0, sizeof(a));
        a.ptrs = ptrs_dev; a.items = its; a.tiles_per_mat = pd.ntiles;
        if (arith == kArithFixed) {
          a.q_in = q_prev;
          a.q_in_stride = q_prev_stride;
          if (!last) {
            a.q_out = reinterpret_cast<int*>(qbase + qoff);
            a.q_out_stride = pd.ntiles;
            qoff += (size_t)pd.ntiles * sizeof(int) * (size_t)hist[n];
            q_prev = a.q_out;
            q_prev_stride = pd.ntiles;
          }
        }
        const double scale = scale_mode ? std::ldexp(1.0, -n) : 1.0;
        pass_scaling(dec, arith, pd, last, scale_mode ? -n : 0, 1.0, scale, &a);
        PassDesc tuned = pd;                   // occupancy override (variants 3 and 4)
        if (pd.D <= 12 && (variants[n] == 3 || variants[n] == 4)) tuned.min_blocks = variants[n] == 3 ? 2 : 3;
        if (launch_pass(arith, dec, tuned, a, pd.ntiles * hist[n], s) != cudaSuccess) return TPD_ERR_CUDA;
      }
      qbase += batched_q_bytes(plan, arith, hist[n]);
    }
    start += hist[n];
  }
  return TPD_OK;
}

}  // namespace
}  // namespace tpd

using namespace tpd;

extern "C" {

void tpd_options_init(tpd_options* opt) {
  if (opt) std::memset(opt, 0, sizeof(*opt));
}

size_t tpd_workspace_size(int n, int dtype, const tpd_options* opt_in) {
  int prec = 0;
  if (check_common(n, dtype, opt_in, &prec) != TPD_OK) return 0;
  const tpd_options eff = effective_options(n, dtype, prec, opt_in);
  const tpd_options* opt = &eff;
  const Plan* plan = get_plan(n, dtype, prec, opt);
  if (!plan) return 0;
  return single_ws(*plan, arith_of(dtype, prec), opt ? (opt->skip_zero != 0) : 0);
}

tpd_status tpd_decompose(void* A, int n, int dtype, const tpd_options* opt, void* workspace,
                         size_t workspace_bytes, void* stream) {
  return single(true, A, n, dtype, 1.0, opt, workspace, workspace_bytes, stream);
}

tpd_status tpd_compose(void* C, int n, int dtype, double scale, const tpd_options* opt, void* workspace,
                       size_t workspace_bytes, void* stream) {
  return single(false, C, n, dtype, scale, opt, workspace, workspace_bytes, stream);
}

tpd_status tpd_decompose_host(const void* A_host, void* W_host, void* dev_A, int n, int dtype,
                              const tpd_options* opt, void* workspace, size_t workspace_bytes, void* stream) {
  int prec = 0;
  tpd_status st = check_common(n, dtype, opt, &prec);
  if (st != TPD_OK) return st;
  if (A_host == nullptr || W_host == nullptr || dev_A == nullptr) return TPD_ERR_INVALID_ARG;
  const size_t align = dtype == TPD_C128 ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(dev_A) % align) return TPD_ERR_MISALIGNED;
  const size_t bytes = ((size_t)1 << (2 * n)) * (dtype == TPD_C128 ? 16 : 8);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(dev_A, A_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return TPD_ERR_CUDA;
  st = single(true, dev_A, n, dtype, 1.0, opt, workspace, workspace_bytes, stream);
  if (st != TPD_OK) return st;
  if (cudaMemcpyAsync(W_host, dev_A, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TPD_ERR_CUDA;
  return TPD_OK;
}

size_t tpd_partial_workspace_size(int n, int dtype, const tpd_options* opt, size_t count) {
  int prec = 0, arith = 0;
  const Plan* plan = nullptr;
  tpd_options eff;
  if (partial_setup(n, dtype, opt, &prec, &arith, &plan, &eff) != TPD_OK) return 0;
  return partial_layout(*plan, arith, count).total;
}

tpd_status tpd_partial_prepare(int n, int dtype, const tpd_options* opt, const unsigned long long* strings,
                               size_t count, void* workspace, size_t workspace_bytes, void* stream) {
  int prec = 0, arith = 0;
  const Plan* plan = nullptr;
  tpd_options eff;
  tpd_status st = partial_setup(n, dtype, opt, &prec, &arith, &plan, &eff);
  if (st != TPD_OK) return st;
  if (count > 0 && strings == nullptr) return TPD_ERR_INVALID_ARG;
  const PartialLayout lay = partial_layout(*plan, arith, count);
  if (workspace == nullptr || workspace_bytes < lay.total) return TPD_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 16) return TPD_ERR_MISALIGNED;
  const unsigned long long nstr = 1ull << (2 * n);
  std::vector<unsigned long long> pos(count);
  for (size_t i = 0; i < count; ++i) {
    if (strings[i] >= nstr) return TPD_ERR_INVALID_ARG;
    pos[i] = rc_of_string(strings[i], n);
  }
  std::vector<std::vector<uint8_t>> need;
  if (plan->npass > 0) partial_need(*plan, pos, &need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  if (count && cudaMemcpyAsync(w, pos.data(), count * sizeof(unsigned long long), cudaMemcpyHostToDevice, s) !=
                   cudaSuccess)
    return TPD_ERR_CUDA;
  for (int p = 0; p < plan->npass; ++p)
    if (cudaMemcpyAsync(w + lay.need_off[p], need[p].data(), need[p].size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return TPD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TPD_ERR_CUDA;   // the host vectors go out of scope
  return TPD_OK;
}

tpd_status tpd_decompose_partial(void* A, int n, int dtype, const tpd_options* opt, size_t count, void* workspace,
                                 size_t workspace_bytes, void* weights, void* stream) {
  int prec = 0, arith = 0;
  const Plan* plan = nullptr;
  tpd_options eff;
  tpd_status st = partial_setup(n, dtype, opt, &prec, &arith, &plan, &eff);
  if (st != TPD_OK) return st;
  if (A == nullptr || (count > 0 && weights == nullptr)) return TPD_ERR_INVALID_ARG;
  const size_t eb = dtype == TPD_C128 ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(A) % eb || reinterpret_cast<uintptr_t>(weights) % eb) return TPD_ERR_MISALIGNED;
  const PartialLayout lay = partial_layout(*plan, arith, count);
  if (workspace == nullptr || workspace_bytes < lay.total) return TPD_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 16) return TPD_ERR_MISALIGNED;
  char* w = static_cast<char*>(workspace);
  const uint8_t* need[kMaxQubits];
  for (int p = 0; p < plan->npass; ++p) need[p] = reinterpret_cast<const uint8_t*>(w + lay.need_off[p]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = run_single(true, arith, A, *plan, 0, 1.0, w + lay.run_off, s, &eff, plan->npass > 0 ? need : nullptr);
  if (st != TPD_OK) return st;
  if (launch_gather(A, reinterpret_cast<const unsigned long long*>(w), count, (int)eb, weights, s) != cudaSuccess)
    return TPD_ERR_CUDA;
  return TPD_OK;
}

size_t tpd_sparse_workspace_size(size_t max_entries) { return sparse_workspace_bytes(max_entries); }

tpd_status tpd_decompose_coo(const int* rows, const int* cols, const void* values, size_t nnz, int n, int dtype,
                             size_t max_entries, unsigned long long* strings, void* weights, size_t capacity,
                             unsigned long long* count, unsigned* status, void* workspace, size_t workspace_bytes,
                             void* stream) {
  if (dtype != TPD_C128) return TPD_ERR_UNSUPPORTED;
  if (n < 1 || n > 15 || count == nullptr || max_entries == 0) return TPD_ERR_INVALID_ARG;
  if (nnz > 0 && (rows == nullptr || cols == nullptr || values == nullptr)) return TPD_ERR_INVALID_ARG;
  if (capacity > 0 && (strings == nullptr || weights == nullptr)) return TPD_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(values) % 16 || reinterpret_cast<uintptr_t>(weights) % 16 ||
      reinterpret_cast<uintptr_t>(strings) % 8 || reinterpret_cast<uintptr_t>(count) % 8 ||
      reinterpret_cast<uintptr_t>(rows) % 4 || reinterpret_cast<uintptr_t>(cols) % 4 ||
      reinterpret_cast<uintptr_t>(status) % 4)
    return TPD_ERR_MISALIGNED;
  if (workspace == nullptr || workspace_bytes < sparse_workspace_bytes(max_entries)) return TPD_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return TPD_ERR_MISALIGNED;
  if (launch_sparse(rows, cols, values, nnz, n, max_entries, strings, weights, capacity, count, workspace, status,
                    static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return TPD_ERR_CUDA;
  return TPD_OK;
}

size_t tpd_nonzero_workspace_size(int n) {
  if (n < 1 || n > kMaxQubits) return 0;
  return nonzero_workspace_bytes(n);
}

tpd_status tpd_nonzero_list(const void* W, int n, int dtype, double tol, unsigned long long* strings,
                            void* weights, size_t capacity, unsigned long long* count, void* workspace,
                            size_t workspace_bytes, void* stream) {
  if (n < 1 || n > kMaxQubits || (dtype != TPD_C128 && dtype != TPD_C64)) return TPD_ERR_INVALID_ARG;
  if (W == nullptr || count == nullptr || !(tol >= 0.0) || (capacity > 0 && (strings == nullptr || weights == nullptr)))
    return TPD_ERR_INVALID_ARG;
  const size_t eb = dtype == TPD_C128 ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(W) % eb || reinterpret_cast<uintptr_t>(weights) % eb ||
      reinterpret_cast<uintptr_t>(strings) % 8 || reinterpret_cast<uintptr_t>(count) % 8)
    return TPD_ERR_MISALIGNED;
  if (workspace == nullptr || workspace_bytes < nonzero_workspace_bytes(n)) return TPD_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return TPD_ERR_MISALIGNED;
  if (launch_nonzero(W, n, (int)eb, tol, strings, weights, capacity, count, workspace,
                     static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return TPD_ERR_CUDA;
  return TPD_OK;
}

tpd_status tpd_convert_layout(const void* src, void* dst, int n, int dtype, int to_string, void* stream) {
  if (n < 1 || n > kMaxQubits || (dtype != TPD_C128 && dtype != TPD_C64)) return TPD_ERR_INVALID_ARG;
  if (src == nullptr || dst == nullptr || (to_string != 0 && to_string != 1)) return TPD_ERR_INVALID_ARG;
  const size_t eb = dtype == TPD_C128 ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(src) % eb || reinterpret_cast<uintptr_t>(dst) % eb) return TPD_ERR_MISALIGNED;
  const size_t bytes = ((size_t)1 << (2 * n)) * eb;
  const uintptr_t a = reinterpret_cast<uintptr_t>(src), b = reinterpret_cast<uintptr_t>(dst);
  if (a < b + bytes && b < a + bytes) return TPD_ERR_INVALID_ARG;
  if (launch_layout(src, dst, n, (int)eb, to_string, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return TPD_ERR_CUDA;
  return TPD_OK;
}

tpd_status tpd_sum_squares(const void* x, size_t count, int dtype, double* result, void* workspace,
                           size_t workspace_bytes, void* stream) {
  if ((dtype != TPD_C128 && dtype != TPD_C64) || result == nullptr || (count > 0 && x == nullptr))
    return TPD_ERR_INVALID_ARG;
  static_assert(TPD_SUMSQ_WORKSPACE_BYTES >= 1024 * sizeof(double), "workspace constant");
  if (workspace == nullptr || workspace_bytes < sumsq_workspace_bytes()) return TPD_ERR_WORKSPACE;
  const size_t eb = dtype == TPD_C128 ? 16 : 8;
  if ((x && reinterpret_cast<uintptr_t>(x) % eb) || reinterpret_cast<uintptr_t>(result) % 8 ||
      reinterpret_cast<uintptr_t>(workspace) % 8)
    return TPD_ERR_MISALIGNED;
  if (launch_sumsq(x, count, (int)eb, result, workspace, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return TPD_ERR_CUDA;
  return TPD_OK;
}

tpd_status tpd_batch_status(const void* workspace, void* stream) {
  if (workspace == nullptr) return TPD_ERR_INVALID_ARG;
  unsigned st = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&st, static_cast<const unsigned*>(workspace) + kCtrlStatus, sizeof(st), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess)
    return TPD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TPD_ERR_CUDA;
  return static_cast<tpd_status>(st);
}

void tpd_test_hold_batch_waits(int on) { g_hold_batch_waits = on != 0; }

size_t tpd_batched_workspace_size(const int* ns, int count, int dtype, const tpd_options* opt) {
  int prec = 0;
  if (check_options(dtype, opt, &prec) != TPD_OK || count < 0 || (count > 0 && ns == nullptr)) return 0;
  int hist[kBatchMaxQubits + 1] = {0};
  for (int i = 0; i < count; ++i) {
    if (ns[i] < 1 || ns[i] > kBatchMaxQubits) return 0;
    hist[ns[i]]++;
  }
  const int arith = arith_of(dtype, prec);
  size_t need = batched_head(count);
  std::vector<const Plan*> plans(kBatchMaxQubits + 1, nullptr);
  for (int n = 1; n <= kBatchMaxQubits; ++n) {
    if (!hist[n]) continue;
    const tpd_options eff = batch_options(n, dtype, prec, opt);
    const Plan* plan = get_plan(n, dtype, prec, &eff);
    if (!plan) return 0;
    plans[n] = plan;
    need += batched_q_bytes(*plan, arith, hist[n]);
  }
  return need + batched_ctrl(hist, plans);
}

tpd_status tpd_decompose_batched(void* const* ptrs_dev, const int* ns_dev, const int* ns, int count, int dtype,
                                 const tpd_options* opt, void* workspace, size_t workspace_bytes, void* stream) {
  return batched(true, ptrs_dev, ns_dev, ns, count, dtype, 0, opt, workspace, workspace_bytes, stream);
}

tpd_status tpd_compose_batched(void* const* ptrs_dev, const int* ns_dev, const int* ns, int count, int dtype,
                               int scale_mode, const tpd_options* opt, void* workspace, size_t workspace_bytes,
                               void* stream) {
  return batched(false, ptrs_dev, ns_dev, ns, count, dtype, scale_mode, opt, workspace, workspace_bytes, stream);
}

tpd_status tpd_tune_set(int n, int dtype, int precision, const tpd_options* tuned) {
  int prec = 0;
  tpd_options probe;
  std::memset(&probe, 0, sizeof(probe));
  probe.precision = precision;
  if (check_common(n, dtype, &probe, &prec) != TPD_OK) return TPD_ERR_INVALID_ARG;
  const auto key = std::make_tuple(n, dtype, prec);
  if (tuned == nullptr) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.erase(key);
    return TPD_OK;
  }
  tpd_options t = *tuned;
  t.precision = precision;
  int p2 = 0;
  if (check_common(n, dtype, &t, &p2) != TPD_OK) return TPD_ERR_INVALID_ARG;
  if (!get_plan(n, dtype, prec, &t)) return TPD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = std::make_tuple(t.tile_bits, t.max_levels, t.variant);
  return TPD_OK;
}

void tpd_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
}

int tpd_plan_describe(int n, int dtype, const tpd_options* opt_in, char* buf, size_t len) {
  int prec = 0;
  if (check_common(n, dtype, opt_in, &prec) != TPD_OK) return -1;
  const tpd_options eff = effective_options(n, dtype, prec, opt_in);
  const Plan* plan = get_plan(n, dtype, prec, &eff);
  if (!plan) return -1;
  std::string s = describe_plan(*plan);
  const L2Chunks ch = l2_chunks(*plan, &eff, eff.skip_zero != 0 || eff.variant == 2);
  if (ch.F >= 2) {
    char tmp[64];
    std::snprintf(tmp, sizeof(tmp), "l2 chunks: passes=%d fixed=", ch.F);
    s += tmp;
    for (size_t k = 0; k < ch.fixed.size(); ++k) {
      std::snprintf(tmp, sizeof(tmp), "%s%d", k ? "," : "", ch.fixed[k]);
      s += tmp;
    }
    s += "\n";
  }
  if (buf && len) {
    std::strncpy(buf, s.c_str(), len - 1);
    buf[len - 1] = 0;
  }
  return plan->npass;
}

const char* tpd_status_string(int status) {
  switch (status) {
    case TPD_OK: return "TPD_OK";
    case TPD_ERR_INVALID_ARG: return "TPD_ERR_INVALID_ARG";
    case TPD_ERR_UNSUPPORTED: return "TPD_ERR_UNSUPPORTED";
    case TPD_ERR_MISALIGNED: return "TPD_ERR_MISALIGNED";
    case TPD_ERR_WORKSPACE: return "TPD_ERR_WORKSPACE";
    case TPD_ERR_CUDA: return "TPD_ERR_CUDA";
    case TPD_ERR_TIMEOUT: return "TPD_ERR_TIMEOUT";
    default: return "TPD_ERR_UNKNOWN";
  }
}

int tpd_version(void) { return 100; }

}  // extern "C"
