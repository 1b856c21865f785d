// Adjoint register kernels with four register qubits per thread (the
// default width), and the dispatch over the widths.
#include "kernels_grad_impl.cuh"

namespace qaoa {

template cudaError_t reg_grad_prepare_r<4>();
template int reg_grad_grid_r<4>(bool, size_t, int);
template cudaError_t launch_reg_grad_r<4>(const RegLaunch &, bool, int, cudaStream_t);

// instantiated in kernels_grad5.cu
extern template cudaError_t reg_grad_prepare_r<5>();
extern template int reg_grad_grid_r<5>(bool, size_t, int);
extern template cudaError_t launch_reg_grad_r<5>(const RegLaunch &, bool, int, cudaStream_t);

cudaError_t reg_grad_prepare() {
    cudaError_t e = reg_grad_prepare_r<4>();
    return e == cudaSuccess ? reg_grad_prepare_r<5>() : e;
}

int reg_grad_grid(bool wide, size_t smem, int p, int rg) {
    return rg == 5 ? reg_grad_grid_r<5>(wide, smem, p) : reg_grad_grid_r<4>(wide, smem, p);
}

cudaError_t launch_reg_grad(const RegLaunch &a, bool wide, int rg, int grid, cudaStream_t s) {
    return rg == 5 ? launch_reg_grad_r<5>(a, wide, grid, s) : launch_reg_grad_r<4>(a, wide, grid, s);
}

}  // namespace qaoa
