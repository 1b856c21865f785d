// Adjoint register kernels with five register qubits per thread (a tuning
// choice: one lane qubit fewer to shuffle, half the resident blocks).
#include "kernels_grad_impl.cuh"

namespace qaoa {

template cudaError_t reg_grad_prepare_r<5>();
template int reg_grad_grid_r<5>(bool, size_t, int);
template cudaError_t launch_reg_grad_r<5>(const RegLaunch &, bool, int, cudaStream_t);

}  // namespace qaoa
