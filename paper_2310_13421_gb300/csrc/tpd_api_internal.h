// Internal interface shared by the C ABI translation units (tpd_api*.cpp):
// option checks, the plan cache and the single-matrix launch sequence.  Host
// code only; not part of the library's interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tpd.h"
#include "tpd_launch.h"
#include "tpd_planner.h"

namespace tpd {
namespace detail {

// arithmetic (kArith*) of a storage type and resolved precision
int arith_of(int dtype, int prec);
// dtype / precision / tuning fields; the resolved precision into *prec
tpd_status check_options(int dtype, const tpd_options* opt, int* prec);
tpd_status check_common(int n, int dtype, const tpd_options* opt, int* prec);
// the caller's options with the tuned defaults filled in (tpd_tune_set)
tpd_options effective_options(int n, int dtype, int prec, const tpd_options* opt);
// cached plan for (n, dtype, precision, tuning fields); nullptr if impossible
const Plan* get_plan(int n, int dtype, int prec, const tpd_options* opt);
size_t align256(size_t b);
// output scaling of pass pd (the 1/2 of Eq. 4, a composition's scale)
void pass_scaling(bool dec, int arith, const PassDesc& pd, bool last, int spow, double sres, double scale,
                  PassArgs* a);
int sm_count();
// workspace bytes of one matrix's plan
size_t single_ws(const Plan& plan, int arith, int skip);
// classes of a pass (binary points it hands on): tiles x 2^(D-K)
size_t class_count(const PassDesc& pd);
// the passes of one matrix, in place; need: per-pass tile masks (partial decomposition) or nullptr
tpd_status run_single(bool dec, int arith, void* mat, const Plan& plan, int skip, double scale, void* ws,
                      cudaStream_t s, const tpd_options* opt, const uint8_t* const* need = nullptr);

}  // namespace detail
}  // namespace tpd
