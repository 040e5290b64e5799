// Launchers for one particle precision; included by kernels_f32.cu and
// kernels_f64.cu, which differ only in T and in their compile flags.
#pragma once
#include <type_traits>

#include "edupic_kernels.cuh"

namespace edupic {

// Calls f(std::integral_constant<int, SH>{}) for the run-time shape index sh.
template <typename F>
static auto with_shape(int sh, F f)
{
    switch (sh) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    default: return f(std::integral_constant<int, 0>{});
    }
}
static_assert(kPushShapeCount == 4, "with_shape covers every shape");

template <typename T>
size_t Launch<T>::push_smem(int nd, int ng_max, int eepf_max, int xt, int shape)
{
    if (xt) return push_smem_bytes<T, true, 0>(nd, ng_max, eepf_max);
    return with_shape(shape, [&](auto sh) { return push_smem_bytes<T, false, decltype(sh)::value>(nd, ng_max, eepf_max); });
}

// Resident blocks per SM of the particle kernel of one species and shape:
// the smaller of its direct-test and null-collision instantiations (one
// grid serves both), for the plain (xt = 0) or the xt-accumulating pair.
template <typename T, int SP, bool XT, int SH>
int blocks_per_sm(size_t smem)
{
    constexpr int nthr = shape_of<T, XT, SH>().threads;
    int a = 0, b = 0;
    cudaFuncSetAttribute(k_push<T, SP, false, XT, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_push<T, SP, true, XT, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_push<T, SP, false, XT, SH>, nthr, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_push<T, SP, true, XT, SH>, nthr, smem);
    int c = a;
    if constexpr (!XT) {
        cudaFuncSetAttribute(k_push<T, SP, false, false, SH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_push<T, SP, false, false, SH, true>, nthr, smem);
    }
    const int m = a < b ? a : b;
    return e == cudaSuccess ? (m < c ? m : c) : -1;
}

template <typename T>
int Launch<T>::push_blocks_per_sm(int species, size_t smem, int xt, int shape)
{
    if (xt) return species == 0 ? blocks_per_sm<T, 0, true, 0>(smem) : blocks_per_sm<T, 1, true, 0>(smem);
    return with_shape(shape, [&](auto sh) {
        constexpr int SH = decltype(sh)::value;
        return species == 0 ? blocks_per_sm<T, 0, false, SH>(smem) : blocks_per_sm<T, 1, false, SH>(smem);
    });
}

template <typename T>
int Launch<T>::push_threads(int xt, int shape)
{
    if (xt) return push_shape_xt<T>().threads;
    return push_shape<T>(shape).threads;
}

template <typename T>
cudaError_t Launch<T>::seed(const DischargeDev *dd, int d, int species, long long n, cudaStream_t st)
{
    k_seed<T><<<1024, 256, 0, st>>>(dd, d, species, n);
    return cudaGetLastError();
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

// null_any: the null-collision instantiation; sorted: the warp-level
// deposition instantiation for discharges in cell order (direct test and no
// xt accumulation only; a sorting discharge with null collisions or xt maps
// runs the plain deposition, which is exact too)
template <typename T, int SP, bool XT, int SH>
cudaError_t push_variant(const DischargeDev *dd, int nd, int measure, int grid, int ng_max, int eb, int null_any,
                         int sorted, size_t smem, cudaStream_t st)
{
    constexpr int nthr = shape_of<T, XT, SH>().threads;
    if (null_any)
        return launch_pdl(k_push<T, SP, true, XT, SH>, dim3(grid), dim3(nthr), smem, st, dd, nd, ng_max, eb, measure);
    if constexpr (!XT)
        if (sorted)
            return launch_pdl(k_push<T, SP, false, false, SH, true>, dim3(grid), dim3(nthr), smem, st, dd, nd, ng_max,
                              eb, measure);
    return launch_pdl(k_push<T, SP, false, XT, SH>, dim3(grid), dim3(nthr), smem, st, dd, nd, ng_max, eb, measure);
}

template <typename T>
cudaError_t Launch<T>::push(const DischargeDev *dd, int nd, int species, int measure, int grid, int ng_max,
                            int eepf_max, int null_any, int xt, int shape, int sorted, cudaStream_t st)
{
    const int eb = species == 0 && measure ? eepf_max : 0;
    const size_t smem = push_smem(nd, ng_max, eb, xt, shape);
    if (xt)
        return species == 0 ? push_variant<T, 0, true, 0>(dd, nd, measure, grid, ng_max, eb, null_any, 0, smem, st)
                            : push_variant<T, 1, true, 0>(dd, nd, measure, grid, ng_max, 0, null_any, 0, smem, st);
    return with_shape(shape, [&](auto sh) {
        constexpr int SH = decltype(sh)::value;
        return species == 0
                   ? push_variant<T, 0, false, SH>(dd, nd, measure, grid, ng_max, eb, null_any, sorted, smem, st)
                   : push_variant<T, 1, false, SH>(dd, nd, measure, grid, ng_max, 0, null_any, sorted, smem, st);
    });
}

template <typename T>
cudaError_t Launch<T>::finalize(const DischargeDev *dd, int nd, int ion_step, int measure, cudaStream_t st)
{
    return launch_pdl(k_finalize<T>, dim3(nd), dim3(kFinalizeThreads), 0, st, dd, nd, ion_step, measure);
}

template <typename T>
cudaError_t Launch<T>::sort(const DischargeDev *dd, int nd, int ng_max, int sms, cudaStream_t st)
{
    constexpr int threads = 256, warps = threads / 32;
    const size_t smem = (size_t)warps * ng_max * 4 + (size_t)(nd + 1) * 4;
    cudaFuncSetAttribute(k_sort_count<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_sort_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e = cudaSuccess;
    for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp) {
        k_sort_count<T><<<2 * sms, threads, smem, st>>>(dd, nd, sp, ng_max);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            k_sort_scan<T><<<nd, threads, (size_t)ng_max * 4, st>>>(dd, sp);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_sort_scatter<T><<<2 * sms, threads, smem, st>>>(dd, nd, sp, ng_max);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_sort_copy<T><<<4 * sms, threads, (size_t)(nd + 1) * 4, st>>>(dd, nd, sp);
            e = cudaGetLastError();
        }
    }
    return e;
}

template <typename T>
cudaError_t Launch<T>::wait_expiry(unsigned long long limit_ns, int *err, cudaStream_t st)
{
    k_wait_expiry<<<1, 32, 0, st>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace edupic
