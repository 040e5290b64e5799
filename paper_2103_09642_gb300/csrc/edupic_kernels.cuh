// Kernels of the PIC/MCC particle loop (Donko et al., arXiv 2103.09642),
// templated on the particle precision T (float or double).
//
//  k_push<T, species>  one pass over the particles of every discharge:
//                      field gather (Sec. 2.1.3) -> leapfrog push (Sec. 2.1.4)
//                      -> electrode absorption (Sec. 2.1.5) -> Monte Carlo
//                      collision (Sec. 2.1.6, Algorithm 6) -> deposition of
//                      the new position for the next step (Sec. 2.1.1).
//  k_finalize<T>       one CTA per discharge: canonical hole fill of absorbed
//                      particles, append of ionisation products, density swap,
//                      diagnostics, and the field solve of the next step
//                      (Sec. 2.1.2, Algorithm 3).
//  k_deposit<T>, k_fields<T>  densities / field after particles are loaded.
//
// The FP64 instantiation is compiled without FMA contraction so that its
// arithmetic matches the plain CPU evaluation of the same expressions.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "edupic_internal.h"

namespace edupic {

#define EDUPIC_QE 1.602176634e-19
#define EDUPIC_ME 9.1093837015e-31
#define EDUPIC_EPS0 8.8541878128e-12
#define EDUPIC_PI 3.14159265358979323846
#define EDUPIC_OPAL_W 10.0

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct VecOf<double> {
    using type = double2;
    static constexpr int n = 2;
};

__device__ __forceinline__ void unpack(const float4 &v, float *a) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ void unpack(const double2 &v, double *a) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ float4 pack(const float *a, float4) { return make_float4(a[0], a[1], a[2], a[3]); }
__device__ __forceinline__ double2 pack(const double *a, double2) { return make_double2(a[0], a[1]); }

// ---------------------------------------------------------------- RNG
// Philox-4x32-10 (Salmon et al., SC'11), counter = (slot, step lo, step hi,
// species << 8 | block), key = seed.
struct Words {
    uint32_t a, b, c, d;
};

__device__ __forceinline__ Words philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Words{c0, c1, c2, c3};
}

struct RngKey {
    uint32_t slot, s_lo, s_hi, k0, k1;
};

// Two uniforms on [0,1): 53-bit in FP64 (words a,b and c,d), 24-bit in FP32
// (words a and c).
__device__ __forceinline__ void uniforms(const Words &w, double &u0, double &u1)
{
    u0 = ((double)(w.a >> 5) * 67108864.0 + (double)(w.b >> 6)) * (1.0 / 9007199254740992.0);
    u1 = ((double)(w.c >> 5) * 67108864.0 + (double)(w.d >> 6)) * (1.0 / 9007199254740992.0);
}
__device__ __forceinline__ void uniforms(const Words &w, float &u0, float &u1)
{
    u0 = (float)(w.a >> 8) * (1.0f / 16777216.0f);
    u1 = (float)(w.c >> 8) * (1.0f / 16777216.0f);
}

template <typename T>
__device__ __forceinline__ void draw(const RngKey &k, int species, int block, T &u0, T &u1)
{
    const Words w = philox(k.slot, k.s_lo, k.s_hi, ((uint32_t)species << 8) | (uint32_t)block, k.k0, k.k1);
    uniforms(w, u0, u1);
}

// Box-Muller pair of standard normals.
template <typename T>
__device__ __forceinline__ void box_muller(T u0, T u1, T &z0, T &z1)
{
    const T r = sqrt((T)-2.0 * log((T)1.0 - u0));
    const T a = (T)(2.0 * EDUPIC_PI) * u1;
    z0 = r * cos(a);
    z1 = r * sin(a);
}

// ---------------------------------------------------------------- helpers
template <typename T>
struct Hot {  // per-discharge constants used for every particle
    T L, inv_dx, dt, factor, n_gas;
    int ng;
};

template <typename T>
__device__ __forceinline__ Hot<T> hot(const DischargeDev &D, int sp)
{
    Hot<T> h;
    if constexpr (std::is_same<T, double>::value) {
        h.L = D.L;
        h.inv_dx = D.inv_dx;
        h.dt = sp == 0 ? D.dt_e : D.dt_i;
        h.factor = sp == 0 ? D.factor_e : D.factor_i;
        h.n_gas = D.n_gas;
    } else {
        h.L = D.Lf;
        h.inv_dx = D.inv_dxf;
        h.dt = sp == 0 ? D.dt_ef : D.dt_if;
        h.factor = sp == 0 ? D.factor_ef : D.factor_if;
        h.n_gas = D.n_gasf;
    }
    h.ng = D.ng;
    return h;
}

// Cell index p and the weight c2 of point p+1 (Sec. 2.1.1 / 2.1.3).  A
// particle at x = L belongs to the last cell with c2 = 1; p is clamped into
// the grid so that no index can leave it.
template <typename T>
__device__ __forceinline__ int cell(T x, T inv_dx, int ng, T &c0)
{
    c0 = x * inv_dx;
    int p = (int)c0;
    p = p < 0 ? 0 : (p > ng - 2 ? ng - 2 : p);
    return p;
}

template <typename T>
__device__ __forceinline__ long long split_q2(T c2);
template <>
__device__ __forceinline__ long long split_q2<double>(double c2)
{
    return __double2ll_rn(c2 * 4294967296.0);
}
template <>
__device__ __forceinline__ long long split_q2<float>(float c2)
{
    return __float2ll_rn(c2 * 4294967296.0f);
}

// Nearest cross-section bin (Algorithm 6).
__device__ __forceinline__ int cs_index(double energy, double de, int n)
{
    const double r = energy / de + 0.5;
    if (!(r < (double)n)) return n - 1;
    const int k = (int)r;
    return k < n - 1 ? k : n - 1;
}
__device__ __forceinline__ int cs_index_f(float energy, float inv_de, int n)
{
    const float r = energy * inv_de + 0.5f;
    if (!(r < (float)n)) return n - 1;
    const int k = (int)r;
    return k < n - 1 ? k : n - 1;
}

// Collision probability P = 1 - exp(-nu dt) (eq. pcoll).  FP32 evaluates the
// same quantity through expm1 to avoid cancellation near 1.
__device__ __forceinline__ double p_coll(double x) { return 1.0 - exp(-x); }
__device__ __forceinline__ float p_coll(float x) { return -expm1f(-x); }

// Euler-angle rotation of Sec. 2.1.6: unit vector of g' for g deflected by
// (chi, eta) given as cosines and sines.
template <typename T>
__device__ __forceinline__ void deflect(T gx, T gy, T gz, T g, T cc, T sc, T ce, T se, T u[3])
{
    const T ct = gx / g;
    const T st = sqrt((T)1.0 - ct * ct);
    T cp, sp;
    if (st == (T)0.0) {
        cp = (T)1.0;
        sp = (T)0.0;
    } else {
        cp = gy / (g * st);
        sp = gz / (g * st);
    }
    u[0] = ct * cc - st * sc * ce;
    u[1] = st * cp * cc + ct * cp * sc * ce - sp * sc * se;
    u[2] = st * sp * cc + ct * sp * sc * ce + cp * sc * se;
}

// e- + Ar (cold gas): returns the process; ionisation fills vej.
template <typename T>
__device__ int collide_electron(const DischargeDev &D, const CsEntry<T> &cs, T &vx, T &vy, T &vz, T u_proc, T u_chi,
                                T u_eta, T u_opal, T vej[3], int &sub)
{
    const T m1 = (T)EDUPIC_ME, m2 = (T)D.ar_mass, ev = (T)EDUPIC_QE, mu = (T)D.mu_e;
    int proc = u_proc < cs.thr1 ? 0 : (u_proc < cs.thr2 ? 1 : 2);
    sub = 0;
    const T gx = vx, gy = vy, gz = vz;
    const T g2 = gx * gx + gy * gy + gz * gz;
    const T g = sqrt(g2);
    const T wx = (m1 * gx) / (m1 + m2), wy = (m1 * gy) / (m1 + m2), wz = (m1 * gz) / (m1 + m2);
    const T eps_c = (T)D.half_mu_e * g2 / ev;
    const T e_exc = (T)D.e_exc, e_ion = (T)D.e_ion;
    if (proc == 1 && eps_c - e_exc < (T)0.0) {
        proc = 0;
        sub = 1;
    }
    if (proc == 2 && eps_c - e_ion < (T)0.0) {
        proc = 0;
        sub = 1;
    }
    T u[3];
    if (proc != 2) {
        T gp = g;
        if (proc == 1) gp = sqrt((T)2.0 * (eps_c - e_exc) * ev / mu);
        const T cc = (T)1.0 - (T)2.0 * u_chi;
        const T sc = sqrt((T)1.0 - cc * cc);
        const T eta = (T)(2.0 * EDUPIC_PI) * u_eta;
        deflect(gx, gy, gz, g, cc, sc, (T)cos(eta), (T)sin(eta), u);
        const T f = m2 / (m1 + m2) * gp;
        vx = wx + f * u[0];
        vy = wy + f * u[1];
        vz = wz + f * u[2];
    } else {
        const T W = (T)EDUPIC_OPAL_W;
        const T avail = eps_c - e_ion;
        const T e_ej = W * tan(u_opal * atan(avail / ((T)2.0 * W)));
        const T e_sc = avail - e_ej;
        const T cs_ = sqrt(e_sc / avail), ss_ = sqrt((T)1.0 - cs_ * cs_);
        const T ce_ = sqrt(e_ej / avail), se_ = sqrt((T)1.0 - ce_ * ce_);
        const T eta = (T)(2.0 * EDUPIC_PI) * u_eta;
        const T cet = cos(eta), set = sin(eta);
        const T gp = sqrt((T)2.0 * e_sc * ev / mu);
        deflect(gx, gy, gz, g, cs_, ss_, cet, set, u);
        const T f = m2 / (m1 + m2) * gp;
        vx = wx + f * u[0];
        vy = wy + f * u[1];
        vz = wz + f * u[2];
        T ue[3];
        deflect(gx, gy, gz, g, ce_, se_, -cet, -set, ue);
        const T vmag = sqrt((T)2.0 * e_ej * ev / m1);
        vej[0] = vmag * ue[0];
        vej[1] = vmag * ue[1];
        vej[2] = vmag * ue[2];
    }
    return proc;
}

// Ar+ + Ar with thermal partner va: 0 isotropic, 1 backward (chi = pi).
template <typename T>
__device__ int collide_ion(const DischargeDev &D, const CsEntry<T> &cs, T &vx, T &vy, T &vz, T vax, T vay, T vaz,
                           T u_proc, T u_chi, T u_eta)
{
    const T m1 = (T)D.ar_mass, m2 = (T)D.ar_mass;
    const int proc = u_proc < cs.thr1 ? 0 : 1;
    const T gx = vx - vax, gy = vy - vay, gz = vz - vaz;
    const T g = sqrt(gx * gx + gy * gy + gz * gz);
    const T wx = (m1 * vx + m2 * vax) / (m1 + m2);
    const T wy = (m1 * vy + m2 * vay) / (m1 + m2);
    const T wz = (m1 * vz + m2 * vaz) / (m1 + m2);
    T cc, sc, ce, se;
    if (proc == 0) {
        cc = (T)1.0 - (T)2.0 * u_chi;
        sc = sqrt((T)1.0 - cc * cc);
        const T eta = (T)(2.0 * EDUPIC_PI) * u_eta;
        ce = cos(eta);
        se = sin(eta);
    } else {
        cc = (T)-1.0;
        sc = (T)0.0;
        ce = (T)1.0;
        se = (T)0.0;
    }
    T u[3];
    deflect(gx, gy, gz, g, cc, sc, ce, se, u);
    const T f = m2 / (m1 + m2) * g;
    vx = wx + f * u[0];
    vy = wy + f * u[1];
    vz = wz + f * u[2];
    return proc;
}

// ---------------------------------------------------------------- block scans
__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive prefix of a per-thread int over the block; returns the prefix,
// writes the block total.  s_w: shared scratch of >= 33 ints.
__device__ __forceinline__ int block_excl_scan(int v, int *s_w, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const int inc = warp_incl_scan(v);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < nw ? s_w[lane] : 0;
        const int wi = warp_incl_scan(w);
        s_w[lane] = wi - w;
        if (lane == 31) s_w[32] = wi;
    }
    __syncthreads();
    const int r = inc - v + s_w[warp];
    total = s_w[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ long long warp_incl_scan64(long long v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ __int128 shfl_up128(__int128 v, int o)
{
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    const unsigned long long l2 = __shfl_up_sync(0xffffffffu, lo, o), h2 = __shfl_up_sync(0xffffffffu, hi, o);
    return (__int128)(((unsigned __int128)h2 << 64) | (unsigned __int128)l2);
}

__device__ __forceinline__ __int128 warp_incl_scan128(__int128 v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const __int128 y = shfl_up128(v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Block exclusive scans of 64-bit and 128-bit integers (exact).
__device__ __forceinline__ long long block_excl_scan64(long long v, long long *s_w, long long &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const long long inc = warp_incl_scan64(v);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const long long w = lane < nw ? s_w[lane] : 0;
        const long long wi = warp_incl_scan64(w);
        s_w[lane] = wi - w;
        if (lane == 31) s_w[32] = wi;
    }
    __syncthreads();
    const long long r = inc - v + s_w[warp];
    total = s_w[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ __int128 block_excl_scan128(__int128 v, __int128 *s_w, __int128 &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const __int128 inc = warp_incl_scan128(v);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const __int128 w = lane < nw ? s_w[lane] : (__int128)0;
        const __int128 wi = warp_incl_scan128(w);
        s_w[lane] = wi - w;
        if (lane == 31) s_w[32] = wi;
    }
    __syncthreads();
    const __int128 r = inc - v + s_w[warp];
    total = s_w[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- particle kernel
template <typename T>
__device__ __forceinline__ const CsEntry<T> *table(const DischargeDev &D, int sp)
{
    return reinterpret_cast<const CsEntry<T> *>(sp == 0 ? D.cs_e : D.cs_i);
}

// Dynamic shared memory layout of k_push: [E: ng_max T][Q: ng_max u64]
// [EEPF: eepf_max u32][tile prefix: nd+1 int].
template <typename T, int SP>
__global__ void __launch_bounds__(kThreads) k_push(const DischargeDev *__restrict__ DD, int nd, int ng_max,
                                                   int eepf_max, int measure)
{
    using V = typename VecOf<T>::type;
    constexpr int VEC = VecOf<T>::n;
    constexpr int TILE = kThreads * VEC;
    extern __shared__ __align__(16) unsigned char smem[];
    T *sE = reinterpret_cast<T *>(smem);
    unsigned long long *sQ = reinterpret_cast<unsigned long long *>(smem + ((ng_max * sizeof(T) + 15) & ~15));
    unsigned int *sH = reinterpret_cast<unsigned int *>(sQ + ng_max);
    int *sPre = reinterpret_cast<int *>(sH + eepf_max);
    __shared__ unsigned int sCnt[EDUPIC_N_COUNTERS];
    __shared__ int sW[33];

    const int tid = threadIdx.x;
    // tiles per discharge -> prefix over discharges (every block computes it)
    {
        int running = 0;
        for (int base = 0; base < nd; base += blockDim.x) {
            const int d = base + tid;
            int cnt = 0;
            if (d < nd && DD[d].active) {
                const long long n = DD[d].ctrl->n[SP];
                cnt = (int)((n + TILE - 1) / TILE);
            }
            int tot;
            const int ex = block_excl_scan(cnt, sW, tot);
            if (d < nd) sPre[d] = running + ex;
            running += tot;
        }
        if (tid == 0) sPre[nd] = running;
    }
    if (tid < EDUPIC_N_COUNTERS) sCnt[tid] = 0;
    __syncthreads();
    const long long total = sPre[nd];
    const long long t0 = (long long)blockIdx.x * total / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * total / gridDim.x;
    if (t0 >= t1) return;

    int cur = -1;
    const DischargeDev *D = nullptr;
    Hot<T> h{};
    long long n = 0;
    RngKey key{};
    const CsEntry<T> *tab = nullptr;
    int cs_n = 0;
    bool eepf_on = false;

    auto flush = [&]() {
        __syncthreads();
        long long *acc = SP == 0 ? D->acc_e : D->acc_i;
        for (int p = tid; p < D->ng; p += blockDim.x) {
            const unsigned long long q = sQ[p];
            if (q) atomicAdd(reinterpret_cast<unsigned long long *>(acc + p), q);
        }
        if (eepf_on) {
            for (int b = tid; b < D->eepf_bins; b += blockDim.x) {
                const unsigned int c = sH[b];
                if (c) atomicAdd(D->eepf + b, (unsigned long long)c);
            }
        }
        if (tid < EDUPIC_N_COUNTERS) {
            const unsigned int c = sCnt[tid];
            if (c) atomicAdd(D->ctrl->counters + tid, (unsigned long long)c);
            sCnt[tid] = 0;
        }
        __syncthreads();
    };

    for (long long t = t0; t < t1; ++t) {
        if (cur < 0 || t >= sPre[cur + 1]) {
            if (cur >= 0) flush();
            ++cur;
            while (sPre[cur + 1] <= t) ++cur;
            D = DD + cur;
            h = hot<T>(*D, SP);
            n = D->ctrl->n[SP];
            const unsigned long long s = (unsigned long long)D->ctrl->step;
            key.s_lo = (uint32_t)s;
            key.s_hi = (uint32_t)(s >> 32);
            key.k0 = (uint32_t)D->seed;
            key.k1 = (uint32_t)(D->seed >> 32);
            tab = table<T>(*D, SP);
            cs_n = SP == 0 ? D->cs_n_e : D->cs_n_i;
            eepf_on = SP == 0 && measure;
            const T *ef = reinterpret_cast<const T *>(D->ef_t);
            for (int p = tid; p < h.ng; p += blockDim.x) {
                sE[p] = ef[p];
                sQ[p] = 0ull;
            }
            if (eepf_on)
                for (int b = tid; b < D->eepf_bins; b += blockDim.x) sH[b] = 0u;
            __syncthreads();
        }
        const long long base = (t - sPre[cur]) * (long long)TILE + (long long)tid * VEC;
        if (base >= n) continue;
        {
            const long long live = n - base < VEC ? n - base : VEC;
            atomicAdd(sCnt + (SP == 0 ? EDUPIC_C_PUSH_E : EDUPIC_C_PUSH_I), (unsigned int)live);
        }

        T *X = reinterpret_cast<T *>(D->x[SP]);
        T *VX = reinterpret_cast<T *>(D->vx[SP]);
        T *VY = reinterpret_cast<T *>(D->vy[SP]);
        T *VZ = reinterpret_cast<T *>(D->vz[SP]);
        T xa[VEC], vxa[VEC], vya[VEC], vza[VEC];
        unpack(*reinterpret_cast<const V *>(X + base), xa);
        unpack(*reinterpret_cast<const V *>(VX + base), vxa);
        unpack(*reinterpret_cast<const V *>(VY + base), vya);
        unpack(*reinterpret_cast<const V *>(VZ + base), vza);

#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const long long slot = base + e;
            if (slot >= n) break;
            const T x = xa[e], vx = vxa[e];
            T vy = vya[e], vz = vza[e];
            // field at the particle (Sec. 2.1.3) and leapfrog push (Sec. 2.1.4)
            T c0;
            const int p = cell<T>(x, h.inv_dx, h.ng, c0);
            const T c1 = (T)(p + 1) - c0, c2 = c0 - (T)p;
            const T e_x = c1 * sE[p] + c2 * sE[p + 1];
            T vxn;
            if (SP == 0)
                vxn = vx - e_x * h.factor;
            else
                vxn = vx + e_x * h.factor;
            if (SP == 0 && eepf_on) {
                // EEPF in the centre 10% with the time-centred velocity
                bool in;
                if constexpr (std::is_same<T, double>::value)
                    in = x >= D->eepf_lo && x <= D->eepf_hi;
                else
                    in = x >= D->eepf_lof && x <= D->eepf_hif;
                if (in) {
                    const T vc = (T)0.5 * (vx + vxn);
                    const T v2c = vc * vc + vy * vy + vz * vz;
                    int b;
                    bool ok;
                    if constexpr (std::is_same<T, double>::value) {
                        const double en = 0.5 * EDUPIC_ME * v2c / EDUPIC_QE;
                        const double r = en / D->eepf_de;
                        ok = r < (double)D->eepf_bins;
                        b = ok ? (int)r : 0;
                    } else {
                        const float r = D->e_of_v2_ef * v2c * D->inv_eepf_def;
                        ok = r < (float)D->eepf_bins;
                        b = ok ? (int)r : 0;
                    }
                    if (ok) atomicAdd(sH + b, 1u);
                }
            }
            const T xn = x + vxn * h.dt;
            xa[e] = xn;
            vxa[e] = vxn;
            const bool inside = (xn >= (T)0.0) && (xn <= h.L);
            if (!inside) {
                // absorption at an electrode (Sec. 2.1.5): record the hole
                const int side = xn < (T)0.0 ? 0 : (xn > h.L ? 1 : -1);
                if (side < 0) {
                    atomicOr(&D->ctrl->error, kErrNan);
                } else {
                    atomicAdd(sCnt + (SP == 0 ? EDUPIC_C_ABS_E_POW : EDUPIC_C_ABS_I_POW) + side, 1u);
                }
                const int hidx = atomicAdd(&D->ctrl->holes[SP], 1);
                if (hidx < kEvents)
                    D->holes[SP][hidx] = (int)slot;
                else
                    atomicOr(&D->ctrl->error, kErrHoles);
                if (SP == 1 && measure && side >= 0) {
                    const T v2 = vxn * vxn + vy * vy + vz * vz;
                    int b;
                    bool ok;
                    if constexpr (std::is_same<T, double>::value) {
                        const double en = D->half_mar * v2 / EDUPIC_QE;
                        const double r = en / D->ifed_de;
                        ok = r < (double)D->ifed_bins;
                        b = ok ? (int)r : 0;
                    } else {
                        const float en = D->e_of_v2_if * v2;
                        const float r = en * D->inv_ifed_def;
                        ok = r < (float)D->ifed_bins;
                        b = ok ? (int)r : 0;
                    }
                    if (ok) atomicAdd((side == 0 ? D->ifed_pow : D->ifed_gnd) + b, 1ull);
                }
                continue;
            }
            key.slot = (uint32_t)slot;
            bool collided = false;
            // ------------------------------------------------ Monte Carlo collision (Algorithm 6)
            if (SP == 0) {
                const T v2 = vxn * vxn + vy * vy + vz * vz;
                const T velocity = sqrt(v2);
                int k;
                if constexpr (std::is_same<T, double>::value) {
                    const double energy = D->half_me * v2 / EDUPIC_QE;
                    k = cs_index(energy, D->cs_de_e, cs_n);
                } else {
                    k = cs_index_f(D->e_of_v2_ef * v2, D->inv_cs_de_ef, cs_n);
                }
                const CsEntry<T> cs = tab[k];
                const T nu = cs.sigsum * h.n_gas * velocity;
                const T pc = p_coll(nu * h.dt);
                T u_test, u_proc;
                draw<T>(key, 0, 0, u_test, u_proc);
                if (u_test < pc) {
                    T u_chi, u_eta, u_opal, u_dummy, vej[3];
                    draw<T>(key, 0, 1, u_chi, u_eta);
                    draw<T>(key, 0, 2, u_opal, u_dummy);
                    T nvx = vxn;
                    int sub;
                    const int proc = collide_electron<T>(*D, cs, nvx, vy, vz, u_proc, u_chi, u_eta, u_opal, vej, sub);
                    vxa[e] = nvx;
                    collided = true;
                    atomicAdd(sCnt + EDUPIC_C_COLL_E_ELA + proc, 1u);
                    if (sub) atomicAdd(sCnt + EDUPIC_C_SUBTHRESHOLD, 1u);
                    if (proc == 2) {
                        T n0, n1, n2, n3, z0, z1, z2, z3;
                        draw<T>(key, 0, 3, n0, n1);
                        draw<T>(key, 0, 4, n2, n3);
                        box_muller(n0, n1, z0, z1);
                        box_muller(n2, n3, z2, z3);
                        const T sth = std::is_same<T, double>::value ? (T)D->sig_th : (T)D->sig_thf;
                        const int pi = atomicAdd(&D->ctrl->products, 1);
                        if (pi < kEvents) {
                            D->prod_parent[pi] = (int)slot;
                            reinterpret_cast<T *>(D->prod_x)[pi] = xn;
                            reinterpret_cast<T *>(D->prod_ve[0])[pi] = vej[0];
                            reinterpret_cast<T *>(D->prod_ve[1])[pi] = vej[1];
                            reinterpret_cast<T *>(D->prod_ve[2])[pi] = vej[2];
                            reinterpret_cast<T *>(D->prod_vi[0])[pi] = sth * z0;
                            reinterpret_cast<T *>(D->prod_vi[1])[pi] = sth * z1;
                            reinterpret_cast<T *>(D->prod_vi[2])[pi] = sth * z2;
                            // the new pair joins the next densities at the parent's x
                            T d0;
                            const int pp = cell<T>(xn, h.inv_dx, h.ng, d0);
                            const long long q2 = split_q2<T>(d0 - (T)pp);
                            atomicAdd(sQ + pp, 4294967296ull - (unsigned long long)q2);
                            atomicAdd(sQ + pp + 1, (unsigned long long)q2);
                            atomicAdd(reinterpret_cast<unsigned long long *>(D->acc_i + pp),
                                      4294967296ull - (unsigned long long)q2);
                            atomicAdd(reinterpret_cast<unsigned long long *>(D->acc_i + pp + 1),
                                      (unsigned long long)q2);
                        } else {
                            atomicOr(&D->ctrl->error, kErrProducts);
                        }
                    }
                }
            } else {
                // thermal partner drawn before the collision probability
                T a0, a1, a2, a3, za, zb, zc, zd;
                draw<T>(key, 1, 0, a0, a1);
                draw<T>(key, 1, 1, a2, a3);
                box_muller(a0, a1, za, zb);
                box_muller(a2, a3, zc, zd);
                T vax, vay, vaz, energy_g2, half;
                int k;
                if constexpr (std::is_same<T, double>::value) {
                    vax = D->sig_th * za;
                    vay = D->sig_th * zb;
                    vaz = D->sig_th * zc;
                    half = D->half_mu_arar;
                } else {
                    vax = D->sig_thf * za;
                    vay = D->sig_thf * zb;
                    vaz = D->sig_thf * zc;
                    half = 0.0f;
                }
                const T gx = vxn - vax, gy = vy - vay, gz = vz - vaz;
                const T g_sqr = gx * gx + gy * gy + gz * gz;
                const T g = sqrt(g_sqr);
                if constexpr (std::is_same<T, double>::value) {
                    energy_g2 = half * g_sqr / EDUPIC_QE;
                    k = cs_index(energy_g2, D->cs_de_i, cs_n);
                } else {
                    k = cs_index_f(D->e_of_g2_if * g_sqr, D->inv_cs_de_if, cs_n);
                }
                const CsEntry<T> cs = tab[k];
                const T nu = cs.sigsum * h.n_gas * g;
                const T pc = p_coll(nu * h.dt);
                T u_test, u_proc;
                draw<T>(key, 1, 2, u_test, u_proc);
                if (u_test < pc) {
                    T u_chi, u_eta;
                    draw<T>(key, 1, 3, u_chi, u_eta);
                    T nvx = vxn;
                    const int proc = collide_ion<T>(*D, cs, nvx, vy, vz, vax, vay, vaz, u_proc, u_chi, u_eta);
                    vxa[e] = nvx;
                    collided = true;
                    atomicAdd(sCnt + EDUPIC_C_COLL_I_ISO + proc, 1u);
                }
            }
            if (collided) {
                VY[slot] = vy;
                VZ[slot] = vz;
            }
            // deposition of the new position for the next step (Sec. 2.1.1)
            T d0;
            const int pp = cell<T>(xn, h.inv_dx, h.ng, d0);
            const long long q2 = split_q2<T>(d0 - (T)pp);
            atomicAdd(sQ + pp, 4294967296ull - (unsigned long long)q2);
            atomicAdd(sQ + pp + 1, (unsigned long long)q2);
        }
        *reinterpret_cast<V *>(X + base) = pack(xa, V{});
        *reinterpret_cast<V *>(VX + base) = pack(vxa, V{});
    }
    if (cur >= 0) flush();
}

// ---------------------------------------------------------------- field solve
// Densities from the fixed-point sums and the Poisson solve for the step whose
// within-cycle index is tc (Algorithm 3).  The tridiagonal system with
// Dirichlet ends is solved through its exact double prefix-sum form: with
// d_p = phi_{p+1} - phi_p, F_p = sum_{k=1..p} D_k, G_p = sum_{j<p} F_j and
// D_k = Q_i,k - Q_e,k (integers), d_p = d_0 - c F_p, phi_p = V + p d_0 - c G_p
// and phi_M = 0 fixes d_0 = (c G_M - V) / M.  F and G are exact integer scans,
// so the result does not depend on the order of summation.
static __device__ void solve_fields(const DischargeDev &D, long long tc)
{
    __shared__ long long sW64[33];
    __shared__ __int128 sW128[33];
    __shared__ double sD[4];
    const int ng = D.ng, M = ng - 1, tid = threadIdx.x, nt = blockDim.x;
    constexpr int PER = (EDUPIC_MAX_GRID + kFinalizeThreads - 1) / kFinalizeThreads;
    // drive voltage V(t)
    double V = 0.0;
    {
        const double t = (double)tc * D.dt_e;
        for (int k = 0; k < D.n_harm; ++k) V += D.harm_volt[k] * cos(2.0 * EDUPIC_PI * D.harm_freq[k] * t);
    }
    // densities (Algorithm 2: x2 at the half-volume edge points)
    for (int p = tid; p < ng; p += nt) {
        double ne = D.factor_w * ((double)D.q_e[p] * (1.0 / 4294967296.0));
        double ni = D.factor_w * ((double)D.q_i[p] * (1.0 / 4294967296.0));
        if (p == 0 || p == ng - 1) {
            ne *= 2.0;
            ni *= 2.0;
        }
        D.n_e[p] = ne;
        D.n_i[p] = ni;
    }
    // F: inclusive scan of D over p = 0..M-1 (D_0 = 0); each thread owns a run
    const int first = tid * PER;
    long long Dv[PER], Fv[PER];
    long long run = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int p = first + j;
        const long long dv = (p >= 1 && p <= M - 1) ? (D.q_i[p] - D.q_e[p]) : 0ll;
        Dv[j] = dv;
        run += dv;
    }
    long long tot64;
    const long long off = block_excl_scan64(run, sW64, tot64);
    long long acc = off;
    __int128 runG = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        acc += Dv[j];
        Fv[j] = acc;
        const int p = first + j;
        if (p <= M - 1) runG += (__int128)acc;
    }
    // G: exclusive scan of F over p = 0..M
    __int128 totG;
    const __int128 offG = block_excl_scan128(runG, sW128, totG);
    if (tid == 0) sD[0] = (D.poisson_c * (double)totG - V) / (double)M;  // d_0
    __syncthreads();
    const double d0 = sD[0], c = D.poisson_c;
    __int128 g = offG;         // G_p for p = first
    long long fprev = off;     // F_{first-1}
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int p = first + j;
        if (p > M) break;
        if (p < M) {
            D.phi[p] = V + (double)p * d0 - c * (double)g;
            g += (__int128)Fv[j];
        } else {
            D.phi[p] = 0.0;
        }
        // E_p = (phi_{p-1} - phi_{p+1}) / (2 dx) = -(d_{p-1} + d_p) / (2 dx) inside;
        // one-sided forms with the half-cell charge at the electrodes
        if (p == 0) {
            const double rho0 = EDUPIC_QE * (D.n_i[0] - D.n_e[0]);
            D.ef[0] = -d0 / D.dx - rho0 * D.dx / (2.0 * EDUPIC_EPS0);
        } else if (p < M) {
            const double dpm1 = d0 - c * (double)fprev, dp = d0 - c * (double)Fv[j];
            D.ef[p] = -(dpm1 + dp) / (2.0 * D.dx);
        } else {
            const double dm1 = d0 - c * (double)fprev;
            const double rhoM = EDUPIC_QE * (D.n_i[M] - D.n_e[M]);
            D.ef[M] = -dm1 / D.dx + rhoM * D.dx / (2.0 * EDUPIC_EPS0);
        }
        fprev = Fv[j];
    }
    __syncthreads();
}

template <typename T>
__device__ void copy_field_t(const DischargeDev &D)
{
    T *et = reinterpret_cast<T *>(D.ef_t);
    for (int p = threadIdx.x; p < D.ng; p += blockDim.x) et[p] = (T)D.ef[p];
}

// ---------------------------------------------------------------- compaction
// Holes of species sp sorted ascending (rank by counting; slots are unique),
// then filled by the tail survivors [N', N) in ascending order.
template <typename T>
__device__ void compact_species(const DischargeDev &D, int sp, int *sA, int *sW, int &H_out, long long &n_out)
{
    Ctrl *C = D.ctrl;
    const long long n = C->n[sp];
    int H = C->holes[sp];
    if (H > kEvents) H = kEvents;  // error bit already set by k_push
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < H; i += nt) sA[i] = D.holes[sp][i];
    __syncthreads();
    constexpr int MAXPER = (kEvents + kFinalizeThreads - 1) / kFinalizeThreads;
    int my_h[MAXPER], my_r[MAXPER];
#pragma unroll
    for (int j = 0; j < MAXPER; ++j) {
        const int i = tid + j * nt;
        my_h[j] = -1;
        my_r[j] = 0;
        if (i < H) {
            const int h = sA[i];
            int r = 0;
            for (int k = 0; k < H; ++k) r += sA[k] < h;
            my_h[j] = h;
            my_r[j] = r;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MAXPER; ++j)
        if (my_h[j] >= 0) sA[my_r[j]] = my_h[j];
    __syncthreads();
    const long long nn = n - H;
    T *X = reinterpret_cast<T *>(D.x[sp]);
    T *VX = reinterpret_cast<T *>(D.vx[sp]);
    T *VY = reinterpret_cast<T *>(D.vy[sp]);
    T *VZ = reinterpret_cast<T *>(D.vz[sp]);
    const T L = std::is_same<T, double>::value ? (T)D.L : (T)D.Lf;
    int filled = 0;
    for (int b = 0; b < H; b += nt) {
        const long long j = nn + b + tid;
        bool alive = false;
        if (b + tid < H) {
            const T xj = X[j];
            alive = (xj >= (T)0.0) && (xj <= L);
        }
        int tot;
        const int r = block_excl_scan(alive ? 1 : 0, sW, tot);
        const int k = filled + r;
        const int dst = (alive && k < H) ? sA[k] : -1;
        if (alive && (dst < 0 || dst >= nn)) atomicOr(&C->error, kErrHoles);  // inconsistent hole list
        if (alive && dst >= 0 && dst < nn) {
            X[dst] = X[j];
            VX[dst] = VX[j];
            VY[dst] = VY[j];
            VZ[dst] = VZ[j];
        }
        filled += tot;
    }
    __syncthreads();
    H_out = H;
    n_out = nn;
}

// Ionisation products appended in ascending parent order.
template <typename T>
__device__ void append_products(const DischargeDev &D, int *sA, long long &ne, long long &ni)
{
    Ctrl *C = D.ctrl;
    int P = C->products;
    if (P > kEvents) P = kEvents;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < P; i += nt) sA[i] = D.prod_parent[i];
    __syncthreads();
    long long room = D.cap[0] - ne;
    if (D.cap[1] - ni < room) room = D.cap[1] - ni;
    const long long keep = (long long)P < room ? (long long)P : (room > 0 ? room : 0);
    T *X0 = reinterpret_cast<T *>(D.x[0]), *X1 = reinterpret_cast<T *>(D.x[1]);
    T *VX0 = reinterpret_cast<T *>(D.vx[0]), *VX1 = reinterpret_cast<T *>(D.vx[1]);
    T *VY0 = reinterpret_cast<T *>(D.vy[0]), *VY1 = reinterpret_cast<T *>(D.vy[1]);
    T *VZ0 = reinterpret_cast<T *>(D.vz[0]), *VZ1 = reinterpret_cast<T *>(D.vz[1]);
    const T *px = reinterpret_cast<const T *>(D.prod_x);
    for (int i = tid; i < P; i += nt) {
        const int h = sA[i];
        int r = 0;
        for (int k = 0; k < P; ++k) r += sA[k] < h;
        if (r < keep) {
            const long long se = ne + r, si = ni + r;
            X0[se] = px[i];
            VX0[se] = reinterpret_cast<const T *>(D.prod_ve[0])[i];
            VY0[se] = reinterpret_cast<const T *>(D.prod_ve[1])[i];
            VZ0[se] = reinterpret_cast<const T *>(D.prod_ve[2])[i];
            X1[si] = px[i];
            VX1[si] = reinterpret_cast<const T *>(D.prod_vi[0])[i];
            VY1[si] = reinterpret_cast<const T *>(D.prod_vi[1])[i];
            VZ1[si] = reinterpret_cast<const T *>(D.prod_vi[2])[i];
        }
    }
    __syncthreads();
    if (tid == 0) {
        C->counters[EDUPIC_C_CREATED] += (unsigned long long)keep;
        if (keep < (long long)P) {
            C->counters[EDUPIC_C_DROPPED] += (unsigned long long)(P - keep);
            C->error |= kErrCapacity;
        }
    }
    ne += keep;
    ni += keep;
}

template <typename T>
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const DischargeDev *__restrict__ DD, int nd,
                                                               int ion_step, int measure)
{
    __shared__ int sA[kEvents];
    __shared__ int sW[33];
    const DischargeDev &D = DD[blockIdx.x];
    if (!D.active) return;
    Ctrl *C = D.ctrl;
    const int tid = threadIdx.x;
    int H;
    long long ne, ni = C->n[1];
    compact_species<T>(D, 0, sA, sW, H, ne);
    if (ion_step) compact_species<T>(D, 1, sA, sW, H, ni);
    append_products<T>(D, sA, ne, ni);
    // grid diagnostics of the step just executed (its densities and potential)
    if (measure) {
        for (int p = tid; p < D.ng; p += blockDim.x) {
            D.sum_ne[p] += D.n_e[p];
            D.sum_ni[p] += D.n_i[p];
            D.sum_phi[p] += D.phi[p];
        }
    }
    const long long next = C->step + 1;
    const long long tc = next % D.nt;
    const bool next_ion = (tc % D.nsub) == 0;
    for (int p = tid; p < D.ng; p += blockDim.x) {
        D.q_e[p] = D.acc_e[p];
        D.acc_e[p] = 0;
        if (next_ion) {
            D.q_i[p] = D.acc_i[p];
            D.acc_i[p] = 0;
        }
    }
    __syncthreads();
    if (tid == 0) {
        C->n[0] = ne;
        C->n[1] = ni;
        C->holes[0] = 0;
        C->holes[1] = 0;
        C->products = 0;
        C->step = next;
        if (measure) C->measured += 1;
    }
    solve_fields(D, tc);
    copy_field_t<T>(D);
}

// Densities of one species from its particles (after a load), into q and,
// for ions between ion steps, also into the pending accumulator.
template <typename T>
__global__ void k_deposit(const DischargeDev *__restrict__ DD, int d, int sp, int also_acc)
{
    const DischargeDev &D = DD[d];
    const long long n = D.ctrl->n[sp];
    const T *X = reinterpret_cast<const T *>(D.x[sp]);
    const T inv_dx = std::is_same<T, double>::value ? (T)D.inv_dx : (T)D.inv_dxf;
    long long *q = sp == 0 ? D.q_e : D.q_i;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        T c0;
        const int p = cell<T>(X[j], inv_dx, D.ng, c0);
        const long long q2 = split_q2<T>(c0 - (T)p);
        atomicAdd(reinterpret_cast<unsigned long long *>(q + p), 4294967296ull - (unsigned long long)q2);
        atomicAdd(reinterpret_cast<unsigned long long *>(q + p + 1), (unsigned long long)q2);
        if (also_acc) {
            atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_i + p), 4294967296ull - (unsigned long long)q2);
            atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_i + p + 1), (unsigned long long)q2);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kFinalizeThreads) k_fields(const DischargeDev *__restrict__ DD, int d)
{
    const DischargeDev &D = DD[d];
    solve_fields(D, D.ctrl->step % D.nt);
    copy_field_t<T>(D);
}

}  // namespace edupic
