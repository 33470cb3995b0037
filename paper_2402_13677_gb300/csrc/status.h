// Status of one linear solve from what its read-back found (host code, no CUDA types, so that
// the mapping can be compiled and checked without a GPU).
#pragma once
#include "../../include/ebit.h"

namespace ebit {

// cuda_ok: the solve's launches and the read-back of its device state succeeded; fault: a
// bounded device wait gave up (every value that launch wrote is then invalid); nonfinite: a
// residual norm was NaN or infinite; converged: every right-hand side reached its tolerance.
inline ebit_status solve_status(bool cuda_ok, bool fault, bool nonfinite, bool converged) {
    if (!cuda_ok || fault) return EBIT_ECUDA;
    if (nonfinite) return EBIT_ENONFINITE;
    return converged ? EBIT_OK : EBIT_ENOCONV;
}

}  // namespace ebit
