// Launchers for one particle precision; included by kernels_f32.cu and
// kernels_f64.cu, which differ only in T and in their compile flags.
#pragma once
#include "edupic_kernels.cuh"

namespace edupic {

template <typename T>
size_t Launch<T>::push_smem(int nd, int ng_max, int eepf_max)
{
    return push_smem_bytes<T>(nd, ng_max, eepf_max);
}

template <typename T>
int Launch<T>::push_blocks_per_sm(int species, size_t smem)
{
    int nb = 0;
    cudaError_t e;
    if (species == 0) {
        cudaFuncSetAttribute(k_push<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<T, 0>, kThreads, smem);
    } else {
        cudaFuncSetAttribute(k_push<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<T, 1>, kThreads, smem);
    }
    return e == cudaSuccess ? nb : -1;
}

template <typename T>
cudaError_t Launch<T>::deposit(const DischargeDev *dd, int nd, int d, int species, int also_acc, cudaStream_t st)
{
    (void)nd;
    k_deposit<T><<<1024, 256, 0, st>>>(dd, d, species, also_acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::fields(const DischargeDev *dd, int nd, int d, cudaStream_t st)
{
    (void)nd;
    k_fields<T><<<1, kGroupB, 0, st>>>(dd, d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::averages(const DischargeDev *dd, int nd, int d, cudaStream_t st)
{
    (void)nd;
    k_averages<T><<<1, kGroupB, 0, st>>>(dd, d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::push(const DischargeDev *dd, int nd, int species, int measure, int grid, int ng_max,
                            int eepf_max, cudaStream_t st)
{
    const size_t smem = push_smem(nd, ng_max, species == 0 && measure ? eepf_max : 0);
    if (species == 0)
        k_push<T, 0><<<grid, kThreads, smem, st>>>(dd, nd, ng_max, species == 0 && measure ? eepf_max : 0, measure);
    else
        k_push<T, 1><<<grid, kThreads, smem, st>>>(dd, nd, ng_max, 0, measure);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::finalize(const DischargeDev *dd, int nd, int ion_step, int measure, cudaStream_t st)
{
    k_finalize<T><<<nd, kFinalizeThreads, 0, st>>>(dd, nd, ion_step, measure);
    return cudaGetLastError();
}

}  // namespace edupic
