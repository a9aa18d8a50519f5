// C ABI of libtpd.so (declared in include/tpd.h), single-matrix calls:
// argument checks, the plan cache, workspace layout and the launch sequence
// of a decomposition or composition, the tuned-default table and the plan
// description.  Host code only; the kernels are behind the launchers of
// tpd_launch.h.  The batched calls live in tpd_api_batched.cpp, the partial
// decomposition, list output, sparse input and layout helpers in
// tpd_api_extra.cpp.
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

#include "tpd_api_internal.h"

namespace tpd {
namespace detail {


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
  if (opt && (opt->variant < 0 || opt->variant > 5)) return TPD_ERR_INVALID_ARG;
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
//   binary points:   one int16 per class of every pass but the last (block
//                    fixed point only): 4^n / 2^K entries for a pass of K levels
size_t class_count(const PassDesc& pd) { return (size_t)pd.ntiles << (pd.D - pd.K); }

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
    for (int i = 0; i + 1 < p.npass; ++i) { L.q_off[i] = off; off += align256(class_count(p.pass[i]) * sizeof(int16_t)); }
  L.q_bytes = off - L.flags_bytes;
  L.total = off;
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
                      cudaStream_t s, const tpd_options* opt, const uint8_t* const* need) {
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
  // with skipping (or a partial decomposition), classes of tiles a pass never
  // visits keep the "zero class" fill
  if ((skip || need) && lay.q_bytes && cudaMemsetAsync(w + lay.flags_bytes, kQFillByte, lay.q_bytes, s) != cudaSuccess)
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
      if (p > 0) a.q_in = reinterpret_cast<const int16_t*>(w + lay.q_off[p - 1]);
      if (!last) a.q_out = reinterpret_cast<int16_t*>(w + lay.q_off[p]);
    }
    pass_scaling(dec, arith, pd, last, spow, sres, scale, &a);
    return a;
  };
  auto tuned_desc = [&](int p) {
    PassDesc tuned = plan.pass[p];            // occupancy override (variants 3 and 4)
    if (tuned.D <= 12 && (variant == 3 || variant == 4)) tuned.min_blocks = variant == 3 ? kOccLow : kOccHigh;
    if (tuned.D > 12 && variant == 1) tuned.min_blocks = 1;   // one 512-thread CTA per tile
    if (variant == 5) tuned.rt_layout = 1;    // layout read at run time
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

}  // namespace detail
}  // namespace tpd

using namespace tpd;
using namespace tpd::detail;

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
