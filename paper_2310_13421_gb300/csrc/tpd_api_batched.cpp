// C ABI of libtpd.so (declared in include/tpd.h): the batched calls -- one
// launch per (qubit count, pass), or the whole batch in one persistent
// launch -- and the batch status word.  Host code only.
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
#include "tpd_shape.h"

namespace tpd {
namespace {
using namespace detail;

// ------------------------------------------------------------------ batched
constexpr int kBatchMaxQubits = kBatchMaxN;
static_assert(kBatchStatusTimeout == TPD_ERR_TIMEOUT && kBatchStatusBadSizes == TPD_ERR_INVALID_ARG,
              "device status codes are tpd_status values");
static_assert(sizeof(BatchParams) <= 32000, "kernel parameter space");

bool g_hold_batch_waits = false;   // test hook (tpd_test_hold_batch_waits)

// workspace: control words (status, work counter, per-matrix pass completion
// counters of the persistent kernel) | items[count] (matrix indices bucketed
// by qubit count, on the device) | bptrs[count] (their pointers, persistent
// form) | per qubit count n (ascending), for the block fixed point: the class
// binary points of hist[n] matrices for every pass but the last
size_t batched_q_bytes(const Plan& plan, int arith, int count_n) {
  if (arith != kArithFixed || plan.npass < 2) return 0;
  size_t b = 0;
  for (int i = 0; i + 1 < plan.npass; ++i) b += class_count(plan.pass[i]) * sizeof(int16_t) * (size_t)count_n;
  return align256(b);
}
size_t batched_ctrl(const int* hist, const std::vector<const Plan*>& plans) {
  size_t words = kCtrlDone;
  for (int n = 1; n <= kBatchMaxQubits; ++n)
    if (hist[n] && plans[n]->npass > 1) words += (size_t)hist[n] * (plans[n]->npass - 1);
  return align256(words * sizeof(unsigned));
}
size_t batched_items_bytes(int count) { return align256((size_t)count * sizeof(int)); }
size_t batched_head(int count) {
  return batched_items_bytes(count) + align256((size_t)count * sizeof(unsigned long long));
}

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
                          unsigned long long* bptrs, char* qbase0, size_t ctrl_bytes, cudaStream_t s) {
  static BatchParams bp;               // large: built under the lock, copied into the launch
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  std::memset(&bp, 0, sizeof(bp));
  bp.count = count;
  for (int n = 0; n <= kBatchMaxQubits; ++n) bp.hist[n] = hist[n];
  bp.scale_mode = dec ? 0 : scale_mode;
  bp.ptrs = ptrs_dev; bp.ns = ns_dev; bp.items = items; bp.bptrs = bptrs; bp.ctrl = ctrl;
  int item_start[kBatchMaxQubits + 2] = {0};
  for (int n = 1; n <= kBatchMaxQubits + 1; ++n) item_start[n] = item_start[n - 1] + hist[n - 1];
  // per n (ascending, as the workspace lays them out): binary-point area and
  // the base of its matrices' completion counters
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
  // claimed items in flight: 2 CTAs per SM, each holding its current and its
  // next item; a matrix's later pass trails its previous pass by at least
  // twice that many items, so the tiles it waits for are done
  const long long inflight = 4ll * sm_count();
  long long first = 1;
  int nseg = 0, ndesc = 0;
  for (int n = kBatchMaxQubits; n >= 7; --n) {
    if (!hist[n]) continue;
    const Plan& p = *plans[n];
    BatchSeg& sg = bp.seg[nseg++];
    sg.kind = kSegPipe; sg.n = n; sg.npass = p.npass; sg.desc = ndesc;
    sg.item_start = item_start[n]; sg.nmat = hist[n];
    sg.tiles = p.pass[0].ntiles;
    // a work item is up to 32 consecutive tiles of one pass of one matrix: the
    // claim, lookups and completion count are paid once per item (GB300,
    // 4096-matrix batch: 11.10 / 10.59 / 10.34 / 10.23 ms for 1 / 4 / 8 / 16
    // tiles; with the later kernels 9.56 / 9.50 / 9.64 ms for 16 / 32 / 64)
    sg.tpi = sg.tiles < kBatchTilesPerItem ? sg.tiles : kBatchTilesPerItem;
    const long long per_round = (long long)p.npass * (sg.tiles / sg.tpi);
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
      sg.shape[i] = (int8_t)(arith == kArithFixed ? match_shape(pd) : -1);
      PassArgs& a = sg.args[i];
      if (arith == kArithFixed) {
        if (i > 0) {
          a.q_in = sg.args[i - 1].q_out;
          a.q_in_stride = (long long)class_count(p.pass[i - 1]);
        }
        if (!last) {
          a.q_out = reinterpret_cast<int16_t*>(qbase0 + qoff);
          a.q_out_stride = (long long)class_count(pd);
          qoff += class_count(pd) * sizeof(int16_t) * hist[n];
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
    sg.first = first; sg.tiles = 1; sg.tpi = 1;
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
  unsigned long long* bptrs =
      reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(items) + batched_items_bytes(count));
  char* qbase = reinterpret_cast<char*>(items) + batched_head(count);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int caller_variant = opt ? opt->variant : 0;
  if (caller_variant == 2 && persistent_fits(hist, plans))
    return run_persistent(dec, arith, ptrs_dev, ns_dev, count, hist, plans, scale_mode, ctrl, items, bptrs, qbase,
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
      const int16_t* q_prev = nullptr;
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
            a.q_out = reinterpret_cast<int16_t*>(qbase + qoff);
            a.q_out_stride = (long long)class_count(pd);
            qoff += class_count(pd) * sizeof(int16_t) * (size_t)hist[n];
            q_prev = a.q_out;
            q_prev_stride = a.q_out_stride;
          }
        }
        const double scale = scale_mode ? std::ldexp(1.0, -n) : 1.0;
        pass_scaling(dec, arith, pd, last, scale_mode ? -n : 0, 1.0, scale, &a);
        PassDesc tuned = pd;                   // occupancy override (variants 3 and 4)
        if (pd.D <= 12 && (variants[n] == 3 || variants[n] == 4)) tuned.min_blocks = variants[n] == 3 ? kOccLow : kOccHigh;
        if (pd.D > 12 && variants[n] == 1) tuned.min_blocks = 1;   // one 512-thread CTA per tile
        if (variants[n] == 5) tuned.rt_layout = 1;                 // layout read at run time
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
using namespace tpd::detail;

extern "C" {

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

}  // extern "C"
