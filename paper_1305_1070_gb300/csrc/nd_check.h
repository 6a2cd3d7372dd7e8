// Input checks of nd_factor / nd_diag_green (nd_check.cu).  Internal.
#pragma once

#include <cuda_runtime.h>

#include "nd_internal.h"

namespace ndgf {

// Relative tolerance of the symmetry and skew-Hermiticity checks.
constexpr double ND_INPUT_TOL = 1e-8;

// Host arrays (NULL = not given): H values symmetric on the pattern and every
// contact block of sigma_r complex symmetric (ND_ERR_NOT_SYMMETRIC).
nd_status host_check_factor(const nd_plan* p, const double* H, const double* sr, int n_e);
// Host arrays: contact blocks of Sigma^< (blocks[0]) and Sigma^> (blocks[1])
// and the phonon diagonals skew-Hermitian (ND_ERR_NOT_SKEW_HERMITIAN).
nd_status host_check_lesser(const nd_plan* p, const double* const blocks[2], const double* const diags[2], int n_e);

// Device arrays: the same checks on the stream; a failure ORs 1 into *flag.
void launch_check_H(const double* H, const int32_t* T, int nnz, int* flag, cudaStream_t s);
void launch_check_blocks(const double* S, int64_t stride, const int64_t* soff, const int32_t* m, int n_contacts,
                         int n_e, bool skew, int* flag, cudaStream_t s);
void launch_check_diag_skew(const double* d, int64_t count, int* flag, cudaStream_t s);

}  // namespace ndgf
