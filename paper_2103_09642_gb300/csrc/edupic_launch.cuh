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
    int nb_nc = 0;
    if (species == 0) {
        cudaFuncSetAttribute(k_push<T, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(k_push<T, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<T, 0, false>, kThreads, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_nc, k_push<T, 0, true>, kThreads, smem);
    } else {
        cudaFuncSetAttribute(k_push<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(k_push<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<T, 1, false>, kThreads, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_nc, k_push<T, 1, true>, kThreads, smem);
    }
    // one grid serves both variants: the smaller resident limit
    return e == cudaSuccess ? (nb < nb_nc ? nb : nb_nc) : -1;
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

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the preceding kernel of the stream finishes; it waits on it
// (griddepcontrol.wait) before touching data.
template <typename K, typename... A>
static cudaError_t launch_pdl(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T>
cudaError_t Launch<T>::push(const DischargeDev *dd, int nd, int species, int measure, int grid, int ng_max,
                            int eepf_max, int null_any, cudaStream_t st)
{
    const int eb = species == 0 && measure ? eepf_max : 0;
    const size_t smem = push_smem(nd, ng_max, eb);
    if (species == 0)
        return null_any ? launch_pdl(k_push<T, 0, true>, dim3(grid), dim3(kThreads), smem, st, dd, nd, ng_max, eb,
                                     measure)
                        : launch_pdl(k_push<T, 0, false>, dim3(grid), dim3(kThreads), smem, st, dd, nd, ng_max, eb,
                                     measure);
    return null_any ? launch_pdl(k_push<T, 1, true>, dim3(grid), dim3(kThreads), smem, st, dd, nd, ng_max, 0, measure)
                    : launch_pdl(k_push<T, 1, false>, dim3(grid), dim3(kThreads), smem, st, dd, nd, ng_max, 0, measure);
}

template <typename T>
cudaError_t Launch<T>::finalize(const DischargeDev *dd, int nd, int ion_step, int measure, cudaStream_t st)
{
    return launch_pdl(k_finalize<T>, dim3(nd), dim3(kFinalizeThreads), 0, st, dd, nd, ion_step, measure);
}

}  // namespace edupic
