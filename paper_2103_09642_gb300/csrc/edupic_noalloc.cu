// Densities and field of given particle positions without any device
// allocation (edupic_fields_noalloc in include/edupic.h).
//
// Some callers cannot allocate device memory in the middle of a run: code
// whose device memory is owned and pre-budgeted by another framework's pool
// (an allocation there would fail or break the budget), or code running
// inside a plugin or a real-time loop that must not touch the allocator (an
// allocation can block on the device or grow the process's footprint).  This
// entry point serves them: the caller passes the particle positions and the
// output arrays, and the only working memory is a fixed array in the
// library's own device image (g_scratch below), which every GPU that loads
// the library holds until the process exits.
//
// Compiled with -fmad=false, like the FP64 particle kernels, so the result
// equals that of edupic_load_particles + edupic_get_fields in FP64 mode.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "edupic_kernels.cuh"

using namespace edupic;

namespace {

// Scratch layout: fixed-point densities Q_e, Q_i and the prefix sums F (each
// EDUPIC_MAX_GRID int64), then the field scalars, the drive voltage and the
// flag of positions outside [0, L].
constexpr size_t kGridBytes = (size_t)EDUPIC_MAX_GRID * sizeof(long long);
constexpr size_t kScratchBytes = 3 * kGridBytes + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static_assert(sizeof(FieldState) + sizeof(double) + sizeof(int) <= 256, "field scalars must fit the scratch tail");

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, never a device address, so it is
// looked up once per device with that device current.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EDUPIC_ECUDA;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return EDUPIC_ECUDA;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return EDUPIC_OK;
}

__global__ void k_na_clear(long long *q, int n, double *vdrive, double v, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) q[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        vdrive[0] = v;
        *bad = 0;
    }
}

// A position outside [0, L] (or not a number) is not deposited: it sets the
// flag, and the call reports EDUPIC_EINVAL.
__global__ void k_na_deposit(const double *__restrict__ x, long long n, double L, double inv_dx, int ng, long long *q,
                             int *bad)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double xj = x[j];
        if (!(xj >= 0.0 && xj <= L)) {
            *bad = 1;
            continue;
        }
        double c0;
        const int p = cell<double>(xj, inv_dx, ng, c0);
        const unsigned long long q2 = split_q2(c0 - (double)p);
        atomicAdd(reinterpret_cast<unsigned long long *>(q + p), 4294967296ull - q2);
        atomicAdd(reinterpret_cast<unsigned long long *>(q + p + 1), q2);
    }
}

__global__ void __launch_bounds__(kGroupB) k_na_solve(DischargeDev D)
{
    __shared__ FieldScratch<kGroupB> sF;
    solve_field<double, kGroupB>(D, 0, false, false, false, true, threadIdx.x, 2, sF);
}

}  // namespace

extern "C" int edupic_fields_noalloc(const edupic_params *p, int64_t step, const double *x_e, int64_t n_e,
                                     const double *x_i, int64_t n_i, double *n_e_out, double *n_i_out,
                                     double *phi_out, double *efield_out, void *cuda_stream)
{
    if (!p || step < 0 || n_e < 0 || n_i < 0 || (n_e > 0 && !x_e) || (n_i > 0 && !x_i)) return EDUPIC_EINVAL;
    if (!n_e_out || !n_i_out || !phi_out || !efield_out) return EDUPIC_EINVAL;
    if (p->n_grid > EDUPIC_MAX_GRID) return EDUPIC_ETOOBIG;
    if (p->n_grid < 3 || !(p->gap_m > 0) || !(p->area_m2 > 0) || !(p->weight >= 0) || p->steps_per_cycle < 1 ||
        !(p->cycle_freq_hz > 0) || p->n_harmonics < 0 || p->n_harmonics > EDUPIC_MAX_HARMONICS)
        return EDUPIC_EINVAL;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *b = static_cast<unsigned char *>(base);
    long long *q_e = reinterpret_cast<long long *>(b);
    long long *q_i = reinterpret_cast<long long *>(b + kGridBytes);
    long long *f = reinterpret_cast<long long *>(b + 2 * kGridBytes);
    FieldState *fs = reinterpret_cast<FieldState *>(b + 3 * kGridBytes);
    double *vdrive = reinterpret_cast<double *>(b + 3 * kGridBytes + sizeof(FieldState));
    int *bad = reinterpret_cast<int *>(b + 3 * kGridBytes + sizeof(FieldState) + sizeof(double));

    // the same derived quantities and drive voltage as the simulation object
    const double kQE = 1.602176634e-19, kEPS0 = 8.8541878128e-12, pi = 3.14159265358979323846;
    DischargeDev D{};
    D.ng = p->n_grid;
    D.nt = 1;
    D.dx = p->gap_m / (p->n_grid - 1);
    D.inv_dx = 1.0 / D.dx;
    D.factor_w = p->weight / (p->area_m2 * D.dx);
    D.poisson_c = D.dx * D.dx * kQE * D.factor_w / (kEPS0 * 4294967296.0);
    D.inv_2dx = 1.0 / (2.0 * D.dx);
    D.edge_c = kQE * D.factor_w * 2.0 / 4294967296.0 * D.dx / (2.0 * kEPS0);
    const double dt_e = 1.0 / (p->cycle_freq_hz * p->steps_per_cycle);
    const double t = (double)(step % p->steps_per_cycle) * dt_e;
    double v = 0.0;
    for (int h = 0; h < p->n_harmonics; ++h) v += p->harm_volt_v[h] * std::cos(2.0 * pi * p->harm_freq_hz[h] * t);
    D.q_e = q_e;
    D.q_i = q_i;
    D.f_cur = f;
    D.fs = fs;
    D.vdrive = vdrive;
    D.n_e = n_e_out;
    D.n_i = n_i_out;
    D.phi = phi_out;
    D.ef = efield_out;
    D.ef_t = efield_out;  // FP64: the particle-precision copy is the field itself

    // every call starts from zeroed densities (the array keeps the last call's contents)
    k_na_clear<<<8, 256, 0, st>>>(q_e, 2 * EDUPIC_MAX_GRID, vdrive, v, bad);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && n_e > 0) k_na_deposit<<<256, 256, 0, st>>>(x_e, n_e, p->gap_m, D.inv_dx, D.ng, q_e, bad);
    if (e == cudaSuccess && n_i > 0) k_na_deposit<<<256, 256, 0, st>>>(x_i, n_i, p->gap_m, D.inv_dx, D.ng, q_i, bad);
    if (e == cudaSuccess) k_na_solve<<<1, kGroupB, 0, st>>>(D);
    if (e == cudaSuccess) e = cudaGetLastError();
    // the flag is read into a stack variable (a pageable copy, no allocation)
    int bad_h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return EDUPIC_ECUDA;
    return bad_h ? EDUPIC_EINVAL : EDUPIC_OK;
}
