// Host-side launchers of the adjoint-gradient kernels.
#pragma once
#include "common.cuh"

namespace helm {

// b = conj(a), n complex entries.
int launch_conj(long long n, const double2* a, double2* b, cudaStream_t s);
// grad += dL/dkappa^2 contribution of one right-hand side (forward field p, adjoint mu).
int launch_gradient(const FineOp& op, const double2* p, const double2* mu, double* grad, cudaStream_t s);

}  // namespace helm
