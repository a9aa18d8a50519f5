// C ABI of libtpd.so (declared in include/tpd.h): the partial decomposition
// of Alg. 3, the paper's list output, sparse (COO) input, layout conversion
// and the sum of squares.  Host code only.
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
namespace {
using namespace detail;

// ------------------------------------------------------------------ partial decomposition
//
// Only the weights of a requested list of strings (Alg. 3: a quaternary
// subtree T of the strings of interest).  The passes run in place as usual,
// but a pass skips every tile that no requested weight depends on.  The
// weight of string t depends, at the input of the pass over levels [b, b+K),
// only on the positions whose bits of every level beta < b already hold t's
// symbol (r_beta, c_beta) and whose bits of every level beta >= b+K satisfy
// r_beta xor c_beta = x_beta(t) (I and Z read the quad's diagonal, X and Y its
// anti-diagonal, Eq. 4): a pass needs the tiles containing such positions,
// enumerated per string (2^(levels after the pass) tile ids at most).  Where
// that enumeration would be longer than the pass has tiles, the pass takes
// instead every tile that shares elements with a needed tile of the pass after
// it (a superset).  Skipped tiles keep what the previous pass left there: the
// later passes read those positions only into weights nobody asked for.  In
// the block fixed point the elements a pass sums together (one class, on one
// binary point) all lie in the same dependency cone, so a needed class never
// contains a skipped position: the requested weights are bit for bit those of
// the full decomposition in every arithmetic, for finite inputs (a tile that
// meets an Inf or NaN anywhere runs the IEEE butterfly).

// workspace: RC positions of the requested strings | per pass, one byte per
// tile: needed | the plan's own workspace (the binary points between passes)
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

// tiles of pass q that share elements with a needed tile of pass q + 1
void closure_need(const PassDesc& a, const PassDesc& b, const std::vector<uint8_t>& need_b,
                  std::vector<uint8_t>* need_a) {
  const unsigned long long C = fixed_mask(a) & fixed_mask(b);
  std::vector<unsigned long long> keys;
  for (unsigned long long t = 0; t < (unsigned long long)b.ntiles; ++t)
    if (need_b[t]) keys.push_back(tile_base_of(b, t) & C);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  for (unsigned long long t = 0; t < (unsigned long long)a.ntiles; ++t)
    (*need_a)[t] = std::binary_search(keys.begin(), keys.end(), tile_base_of(a, t) & C) ? 1 : 0;
}

void partial_need(const Plan& plan, int n, const std::vector<unsigned long long>& pos,
                  std::vector<std::vector<uint8_t>>* need) {
  const int P = plan.npass;
  need->assign(P, {});
  for (int p = 0; p < P; ++p) (*need)[p].assign((size_t)plan.pass[p].ntiles, 0);
  for (int p = P - 1; p >= 0; --p) {
    const PassDesc& pd = plan.pass[p];
    // tile-id position of each global bit (-1: a bit of the tile)
    int at[2 * kMaxQubits];
    for (int g = 0; g < 2 * n; ++g) at[g] = -1;
    for (int j = 0; j < pd.nrest; ++j) at[pd.rest_gbit[j]] = j;
    std::vector<int> future;                 // levels after the pass with a bit outside the tile
    for (int beta = pd.b + pd.K; beta < n; ++beta)
      if (at[beta] >= 0 || at[n + beta] >= 0) future.push_back(beta);
    const unsigned long long per = 1ull << future.size();
    if (p < P - 1 && (unsigned long long)pos.size() * per > 4ull * (unsigned long long)pd.ntiles) {
      closure_need(pd, plan.pass[p + 1], (*need)[p + 1], &(*need)[p]);
      continue;
    }
    for (unsigned long long x : pos) {
      unsigned long long base = 0;           // the levels before the pass: t's symbol bits
      for (int beta = 0; beta < pd.b; ++beta) {
        if (at[beta] >= 0) base |= ((x >> beta) & 1ull) << at[beta];
        if (at[n + beta] >= 0) base |= ((x >> (n + beta)) & 1ull) << at[n + beta];
      }
      for (unsigned long long f = 0; f < per; ++f) {
        unsigned long long t = base;
        for (size_t i = 0; i < future.size(); ++i) {
          const int beta = future[i];
          const unsigned long long r = (f >> i) & 1ull;
          const unsigned long long c = r ^ (((x >> beta) ^ (x >> (n + beta))) & 1ull);
          if (at[n + beta] >= 0) t |= r << at[n + beta];
          if (at[beta] >= 0) t |= c << at[beta];
        }
        (*need)[p][t] = 1;
      }
    }
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

}  // namespace
}  // namespace tpd

using namespace tpd;
using namespace tpd::detail;

extern "C" {

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
  if (plan->npass > 0) partial_need(*plan, n, pos, &need);
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

}  // extern "C"
