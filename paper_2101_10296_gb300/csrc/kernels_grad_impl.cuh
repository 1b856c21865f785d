// Adjoint instantiations of the register-resident cone kernel for one
// register width RG (included by kernels_grad.cu, RG = 4, and
// kernels_grad5.cu, RG = 5, which compile in parallel): the depth p is a
// compile-time constant for p = 1, 2, 3 (layer loops fully unrolled), read
// at run time otherwise.
#pragma once

#include "cone_kernel.cuh"

namespace qaoa {

int occupancy_grid(const void *fn, int block, size_t smem);

namespace {

template <int RG, typename MT, int PC>
const void *grad_fn() {
    return (const void *)reg_cone_kernel<RG, MT, true, PC>;
}

template <int RG, typename MT>
const void *grad_fn_for(int p) {
    switch (p) {
        case 1: return grad_fn<RG, MT, 1>();
        case 2: return grad_fn<RG, MT, 2>();
        case 3: return grad_fn<RG, MT, 3>();
        default: return grad_fn<RG, MT, 0>();
    }
}

template <int RG, typename MT, int PC>
void launch(const RegLaunch &a, int grid, size_t sm, cudaStream_t s) {
    reg_cone_kernel<RG, MT, true, PC><<<grid, kRegBlock, sm, s>>>(a);
}

template <int RG, typename MT>
void launch_for(const RegLaunch &a, int grid, size_t sm, cudaStream_t s) {
    switch (a.p) {
        case 1: launch<RG, MT, 1>(a, grid, sm, s); break;
        case 2: launch<RG, MT, 2>(a, grid, sm, s); break;
        case 3: launch<RG, MT, 3>(a, grid, sm, s); break;
        default: launch<RG, MT, 0>(a, grid, sm, s); break;
    }
}

}  // namespace

template <int RG>
cudaError_t reg_grad_prepare_r() {
    cudaError_t e = cudaSuccess;
    for (int p = 0; p <= 3 && e == cudaSuccess; ++p) {
        for (int w = 0; w < 2 && e == cudaSuccess; ++w)
            e = cudaFuncSetAttribute(w ? grad_fn_for<RG, uint64_t>(p) : grad_fn_for<RG, uint32_t>(p),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kRegMaxSmem);
    }
    return e;
}

template <int RG>
int reg_grad_grid_r(bool wide, size_t smem, int p) {
    return occupancy_grid(wide ? grad_fn_for<RG, uint64_t>(p) : grad_fn_for<RG, uint32_t>(p), kRegBlock, smem);
}

template <int RG>
cudaError_t launch_reg_grad_r(const RegLaunch &a, bool wide, int grid, cudaStream_t s) {
    const size_t sm = reg_smem_bytes(a.jpt, a.p, a.cmax1, true);
    if (wide)
        launch_for<RG, uint64_t>(a, grid, sm, s);
    else
        launch_for<RG, uint32_t>(a, grid, sm, s);
    return cudaGetLastError();
}

}  // namespace qaoa
