// Kernels of the PIC/MCC particle loop (Donko et al., arXiv 2103.09642),
// templated on the particle precision T (float or double).
//
//  k_push<T, species>  one pass over the particles of every discharge:
//                      field gather (Sec. 2.1.3) -> leapfrog push (Sec. 2.1.4)
//                      -> electrode absorption (Sec. 2.1.5) -> Monte Carlo
//                      collision (Sec. 2.1.6, Algorithm 6) -> deposition of
//                      the new position for the next step (Sec. 2.1.1).
//  k_finalize<T>       one CTA per discharge, two warp groups working at once:
//                      (A) canonical hole fill of absorbed particles and
//                      append of ionisation products; (B) density swap,
//                      diagnostics and the field solve of the next step
//                      (Sec. 2.1.2, Algorithm 3).
//  k_deposit<T>, k_fields<T>  densities / field after particles are loaded.
//
// The FP64 instantiation is compiled without FMA contraction so that its
// arithmetic matches the plain CPU evaluation of the same expressions.
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <type_traits>

#include "edupic_internal.h"

namespace edupic {

#define EDUPIC_QE 1.602176634e-19
#define EDUPIC_ME 9.1093837015e-31
#define EDUPIC_EPS0 8.8541878128e-12
#define EDUPIC_PI 3.14159265358979323846
#define EDUPIC_OPAL_W 10.0
#ifndef EDUPIC_PUSH_MIN_BLOCKS
#define EDUPIC_PUSH_MIN_BLOCKS 2  // resident FP32 particle-kernel blocks per SM the register budget targets
#endif

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    using type = float4;
    using pair = float2;
    static constexpr int n = 4;
};
template <>
struct VecOf<double> {
    using type = double2;
    using pair = double2;
    static constexpr int n = 2;
};

__device__ __forceinline__ void unpack(const float4 &v, float *a) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ void unpack(const double2 &v, double *a) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ float4 pack(const float *a, float4) { return make_float4(a[0], a[1], a[2], a[3]); }
__device__ __forceinline__ double2 pack(const double *a, double2) { return make_double2(a[0], a[1]); }

template <typename T>
__host__ __device__ constexpr bool is_f64() { return std::is_same<T, double>::value; }

// a * b + c.  FP32: one fused rounding (fmaf).  FP64: two roundings, the
// plain CPU evaluation of the same expression (the FP64 kernels match the
// oracle).  Both units are compiled without automatic contraction, so every
// fused operation is one of these, and each launch shape of a kernel rounds
// exactly as the others do.
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return a * b + c; }

// Paired FP32 arithmetic (sm_100+ f32x2 instructions): two independent
// lanes in one instruction, each rounded exactly as the scalar operation
// (round to nearest, denormals flushed, as the FP32 unit is compiled).
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.ftz.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.ftz.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c)  // a * b + c, one rounding
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.ftz.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 f2_sq3(float2 x, float2 y, float2 z)  // sq3 of two lanes
{
    return f2_fma(z, z, f2_fma(y, y, f2_mul(x, x)));
}

// v_x^2 + v_y^2 + v_z^2, summed left to right
template <typename T>
__device__ __forceinline__ T sq3(T x, T y, T z)
{
    return madd(z, z, madd(y, y, x * x));
}

// ---------------------------------------------------------------- RNG
// Philox-4x32-10 (Salmon et al., SC'11).  Counter (c0, step lo, step hi,
// species << 8 | block), key = seed.  Block 0 holds collision-test uniforms:
// in FP64 with c0 = slot / 2 (53 bits from words a,b for even slots, c,d for
// odd), in FP32 with c0 = slot / 4 (24 bits from word slot % 4).  Blocks >= 1
// with c0 = slot hold a particle's other draws.
struct Words {
    uint32_t a, b, c, d;
};

// 32 x 32 -> 64-bit product as its (lo, hi) words, one wide multiply.
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi)
{
    asm("{\n\t.reg .u64 t;\n\tmul.wide.u32 t, %2, %3;\n\tmov.b64 {%0, %1}, t;\n\t}"
        : "=r"(lo), "=r"(hi)
        : "r"(a), "r"(b));
}

__device__ __forceinline__ Words philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0, hi0, lo1, hi1;
        mul_wide(0xD2511F53u, c0, lo0, hi0);
        mul_wide(0xCD9E8D57u, c2, lo1, hi1);
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

// The same block with the ten round keys (k0, k1 of rounds 2j and 2j + 1 in
// rk[j]) read from shared memory, where they are formed once per discharge.
__device__ __forceinline__ Words philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint4 *rk)
{
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const uint4 k = rk[j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t lo0, hi0, lo1, hi1;
            mul_wide(0xD2511F53u, c0, lo0, hi0);
            mul_wide(0xCD9E8D57u, c2, lo1, hi1);
            const uint32_t n0 = hi1 ^ c1 ^ (h ? k.z : k.x), n2 = hi0 ^ c3 ^ (h ? k.w : k.y);
            c0 = n0;
            c1 = lo1;
            c2 = n2;
            c3 = lo0;
        }
    }
    return Words{c0, c1, c2, c3};
}

struct RngKey {
    uint32_t s_lo, s_hi, k0, k1;
};

__device__ __forceinline__ double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}
__device__ __forceinline__ float u24(uint32_t a) { return (float)(a >> 8) * (1.0f / 16777216.0f); }

__device__ __forceinline__ void uniforms(const Words &w, double &u0, double &u1)
{
    u0 = u53(w.a, w.b);
    u1 = u53(w.c, w.d);
}
__device__ __forceinline__ void uniforms(const Words &w, float &u0, float &u1)
{
    u0 = u24(w.a);
    u1 = u24(w.c);
}

// Per-particle block b >= 1 of slot `slot`.
template <typename T>
__device__ __forceinline__ void draw(const RngKey &k, uint32_t slot, int species, int block, T &u0, T &u1)
{
    const Words w = philox(slot, k.s_lo, k.s_hi, ((uint32_t)species << 8) | (uint32_t)block, k.k0, k.k1);
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
// Cell index p and c0 = x / dx (Sec. 2.1.1 / 2.1.3).  A particle at x = L
// belongs to the last cell; p is clamped into the grid so that no index can
// leave it.
template <typename T>
__device__ __forceinline__ int cell(T x, T inv_dx, int ng, T &c0)
{
    c0 = x * inv_dx;
    // one unsigned minimum: c0 in (-1, 0] truncates to 0, anything below -1
    // (no particle inside the gap) wraps above ng - 2 and clamps there
    return (int)min((unsigned)(int)c0, (unsigned)(ng - 2));
}

// Fixed-point weight of point p+1: round-to-nearest-even(c2 * 2^32).
__device__ __forceinline__ unsigned long long split_q2(double c2)
{
    return (unsigned long long)__double2ll_rn(c2 * 4294967296.0);
}
__device__ __forceinline__ unsigned long long split_q2(float c2)
{
    // c2 < 1 in FP32 means c2 <= 1 - 2^-24, so c2 * 2^32 < 2^32 fits 32 bits
    return c2 < 1.0f ? (unsigned long long)__float2uint_rn(c2 * 4294967296.0f) : 4294967296ull;
}

// Per-block deposition accumulator in shared memory.  A particle in cell p
// adds q1 = 2^32 - q2 to point p and q2 to point p+1; the block keeps, per
// cell, the count and the sum S_p of q2 in two 16-bit halves (three 32-bit
// shared atomics per deposit; measured faster on sm_103a than one packed
// 64-bit shared atomic), and forms Q_p = 2^32 cnt_p - S_p + S_{p-1} when it
// flushes.  The halves cannot overflow while a cell takes fewer than 2^16
// deposits between flushes: the kernel flushes every kDepFlush particles,
// a flush interval holds at most kDepFlush + one tile particles, and each
// takes one deposit (ionisation products and emitted electrons deposit
// straight into the discharge's global accumulators).
struct DepAcc {
    unsigned int *cnt, *lo, *hi;
    uint32_t s_cnt, s_lo, s_hi;  // the same arrays as shared-memory addresses
};
constexpr int kDepFlush = 64000;
static_assert(kDepFlush + 1024 < 65536, "a flush interval stays below 2^16 deposits per cell");

// Reduction into shared memory in the shared state space (no generic
// address resolution, and no ordering against global accesses).
__device__ __forceinline__ void red_shared_u32(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ void dep_add(const DepAcc &a, int p, unsigned long long q2)
{
    red_shared_u32(a.s_cnt + 4u * (uint32_t)p, 1u);
    red_shared_u32(a.s_lo + 4u * (uint32_t)p, (unsigned int)(q2 & 0xFFFFull));
    red_shared_u32(a.s_hi + 4u * (uint32_t)p, (unsigned int)(q2 >> 16));
}

// The same deposit when c holds: one predicate for the three reductions, so
// no branch is taken around them.
__device__ __forceinline__ void dep_add_if(const DepAcc &a, int p, unsigned long long q2, bool c)
{
    const uint32_t o = 4u * (uint32_t)p;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %6, 0;\n\t@q red.shared.add.u32 [%0], %3;\n\t"
        "@q red.shared.add.u32 [%1], %4;\n\t@q red.shared.add.u32 [%2], %5;\n\t}" ::"r"(a.s_cnt + o),
        "r"(a.s_lo + o), "r"(a.s_hi + o), "r"(1u), "r"((unsigned int)(q2 & 0xFFFFull)), "r"((unsigned int)(q2 >> 16)),
        "r"((unsigned)c));
}

__device__ __forceinline__ unsigned long long dep_cnt(const DepAcc &a, int p) { return a.cnt[p]; }
__device__ __forceinline__ unsigned long long dep_sum(const DepAcc &a, int p)  // S_p
{
    return (unsigned long long)a.lo[p] + ((unsigned long long)a.hi[p] << 16);
}

// Bucket of a squared speed for the electrons' collision bound: the
// exponent and the top five mantissa bits of its floating-point form (32
// buckets per octave, monotonic in v^2 >= 0), clamped into the table's
// [base, base + n - 1]; the last bucket is unbounded.
__device__ __forceinline__ int lv_bucket(float w2, int base, int n)
{
    const int b = (int)(__float_as_uint(w2) >> 18);
    return min(max(b, base), base + n - 1) - base;
}
__device__ __forceinline__ int lv_bucket(double w2, int base, int n)
{
    const int b = (int)((unsigned long long)__double_as_longlong(w2) >> 47);
    return min(max(b, base), base + n - 1) - base;
}

// Nearest cross-section bin (Algorithm 6).
__device__ __forceinline__ int cs_index(double energy, double de, int n)
{
    const double r = energy / de + 0.5;
    if (!(r < (double)n)) return n - 1;
    const int k = (int)r;
    return k < n - 1 ? k : n - 1;
}
__device__ __forceinline__ int cs_index_f(float r, int n)  // r = energy / de + 0.5 >= 0.5 already formed
{
    const int k = (int)r;  // saturating conversion: huge r gives INT_MAX
    return k < n - 1 ? k : n - 1;
}

// Collision probability P = 1 - exp(-x), x = nu dt (eq. pcoll).  FP32 uses
// the Taylor series of 1 - e^-x below x = 1/8 (truncation below 1e-7
// relative) to avoid the cancellation of 1 - exp near 1.
__device__ __forceinline__ double p_coll(double x) { return 1.0 - exp(-x); }
__device__ __forceinline__ float p_coll(float x)
{
    const float series =
        x * madd(-x, madd(-x, madd(-x, madd(-x, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f), 0.5f), 1.0f);
    const float direct = 1.0f - __expf(-x);
    return x < 0.125f ? series : direct;
}

// Euler-angle rotation of Sec. 2.1.6: unit vector of g' for g deflected by
// (chi, eta) given as cosines and sines.
template <typename T>
__device__ __forceinline__ void deflect(T gx, T gy, T gz, T g, T cc, T sc, T ce, T se, T u[3])
{
    const T ct = gx / g;
    const T st = sqrt(gy * gy + gz * gz) / g;  // well conditioned when g is nearly along x
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
__device__ __forceinline__ int collide_electron(const DischargeDev &D, T thr1, T thr2, T &vx, T &vy, T &vz, T u_proc,
                                                T u_chi, T u_eta, T u_opal, T vej[3], int &sub)
{
    const T m1 = (T)EDUPIC_ME, m2 = (T)D.ar_mass, ev = (T)EDUPIC_QE, mu = (T)D.mu_e;
    int proc = u_proc < thr1 ? 0 : (u_proc < thr2 ? 1 : 2);
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
__device__ __forceinline__ int collide_ion(const DischargeDev &D, T thr1, T &vx, T &vy, T &vz, T vax, T vay, T vaz,
                                           T u_proc, T u_chi, T u_eta)
{
    const T m1 = (T)D.ar_mass, m2 = (T)D.ar_mass;
    const int proc = u_proc < thr1 ? 0 : 1;
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

// ---------------------------------------------------------------- scans
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// Programmatic dependent launch: wait until the preceding kernel of the
// stream has completed and its writes are visible; allow the following
// kernel to be scheduled (it waits the same way before touching data).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------- mbarrier wait
// A bounded wait on an mbarrier phase (used by the self-test of the expiry
// path; the particle kernel itself waits only for its own copies).
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier for at most limit_ns (one second by
// default); false if the wait expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// Test of the bounded wait: one block waits on a barrier that nothing ever
// arrives on, so every wait expires after limit_ns; the block records the
// expiry in *err (kErrTimeout) and returns.
static __global__ void k_wait_expiry(unsigned long long limit_ns, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(err, kErrTimeout);
}

// Per-thread asynchronous copies global -> shared of 16 bytes (cp.async,
// bypassing L1), grouped per tile: a thread waits only for its own groups.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename V>
__device__ __forceinline__ V warp_incl_scan(V v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive prefix of a per-thread value over a group of g threads (whole
// warps, group-local id gtid) synchronised by named barrier `bar`.  Returns
// the prefix and writes the group total.  s_w: shared scratch of >= 33 V.
template <typename V>
__device__ __forceinline__ V group_excl_scan(V v, V *s_w, V &total, int gtid, int g, int bar)
{
    const int lane = gtid & 31, warp = gtid >> 5, nw = g >> 5;
    const V inc = warp_incl_scan(v);
    if (lane == 31) s_w[warp] = inc;
    bar_sync(bar, g);
    if (warp == 0) {
        const V w = lane < nw ? s_w[lane] : (V)0;
        const V wi = warp_incl_scan(w);
        s_w[lane] = wi - w;
        if (lane == 31) s_w[32] = wi;
    }
    bar_sync(bar, g);
    const V r = inc - v + s_w[warp];
    total = s_w[32];
    bar_sync(bar, g);
    return r;
}

// ---------------------------------------------------------------- int128 reduction
__device__ __forceinline__ __int128 shfl_down128(__int128 v, int o)
{
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
    const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, o), h2 = __shfl_down_sync(0xffffffffu, hi, o);
    return (__int128)(((unsigned __int128)h2 << 64) | (unsigned __int128)l2);
}

// Exact sum of a per-thread int128 over a group of g threads; every thread
// gets the total.  s_w: shared scratch of >= 32 int128.
__device__ __forceinline__ __int128 group_sum128(__int128 v, __int128 *s_w, int gtid, int g, int bar)
{
    const int lane = gtid & 31, warp = gtid >> 5, nw = g >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_down128(v, o);
    if (lane == 0) s_w[warp] = v;
    bar_sync(bar, g);
    __int128 t = 0;
    for (int w = 0; w < nw; ++w) t += s_w[w];
    bar_sync(bar, g);
    return t;
}

// ---------------------------------------------------------------- colliders
// Collisions are rare (P_coll ~ 1e-3), so the particle loop only queues the
// slots whose test passed; a separate section of the kernel then executes
// them (Algorithm 6 after the test).  It re-derives the table index and, for
// Ar+, the thermal partner from the same counter-based draws, so the result
// is the same as executing the collision in place.
constexpr int kWarpQueue = 512;  // queued colliders per warp before the warp drains them

// Null-collision method (Sec. 2.1.6): a particle picked by its test uniform
// u < P* collides for real when u / P* < nu / nu* (given the pick, u / P* is
// uniform on [0, 1)), nu = n sigma_tot(k) q with q the speed (e-) or
// relative speed (Ar+) whose square is q2.  Counts nu > nu* (an energy past
// the table).
template <typename T, int SP>
__device__ __forceinline__ bool null_real(const DischargeDev &D, int k, T q2, T u, unsigned int *sCnt)
{
    const T sg = reinterpret_cast<const T *>(D.cs_sig[SP])[k];
    bool over, real;
    if constexpr (is_f64<T>()) {
        const double nu = sg * D.n_gas * sqrt(q2);
        over = nu > D.nu_star[SP];
        real = u / D.p_star[SP] < nu / D.nu_star[SP];
    } else {
        const float r = sg * sqrtf(q2) * D.null_ratf[SP];
        over = r > 1.0f;
        real = u < r * D.p_starf[SP];
    }
    if (over) atomicAdd(sCnt + EDUPIC_C_NULL_OVER, 1u);
    return real;
}

// The same decision with sigma_tot of the entry already fetched (sg).
template <typename T, int SP>
__device__ __forceinline__ bool null_real_sg(const DischargeDev &D, T sg, T q2, T u, unsigned int *sCnt)
{
    bool over, real;
    if constexpr (is_f64<T>()) {
        const double nu = sg * D.n_gas * sqrt(q2);
        over = nu > D.nu_star[SP];
        real = u / D.p_star[SP] < nu / D.nu_star[SP];
    } else {
        const float r = sg * sqrtf(q2) * D.null_ratf[SP];
        over = r > 1.0f;
        real = u < r * D.p_starf[SP];
    }
    if (over) atomicAdd(sCnt + EDUPIC_C_NULL_OVER, 1u);
    return real;
}

// *p += 1 (64-bit, global memory) when c holds: a predicated reduction in
// the global state space, so that the compiler may keep shared-memory
// accesses of neighbouring particles on either side of it.
__device__ __forceinline__ void red_add1_global_if(unsigned long long *p, bool c)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t@q red.relaxed.gpu.global.add.u64 [%0], %2;\n\t}" ::"l"(
                     __cvta_generic_to_global(p)),
                 "r"((unsigned)c), "l"(1ull));
}

// Read-only load of *p when c holds (a predicated load: the address is not
// touched otherwise), else 0.  Issued early so that its latency overlaps
// the work before its use.
__device__ __forceinline__ float ldg_if(const float *p, bool c)
{
    float v = 0.0f;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.f32 %0, [%1];\n\t}"
        : "+f"(v)
        : "l"(p), "r"((unsigned)c));
    return v;
}
__device__ __forceinline__ double ldg_if(const double *p, bool c)
{
    double v = 0.0;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.f64 %0, [%1];\n\t}"
        : "+d"(v)
        : "l"(p), "r"((unsigned)c));
    return v;
}

// Collision-test uniform of `slot` for species SP: word slot % VEC of the
// block-0 Philox draw of its group of VEC slots (the draw of the particle loop).
template <typename T, int SP>
__device__ __forceinline__ T test_uniform(const RngKey &key, uint32_t slot)
{
    constexpr uint32_t VEC = VecOf<T>::n;
    const Words w = philox(slot / VEC, key.s_lo, key.s_hi, (uint32_t)SP << 8, key.k0, key.k1);
    if constexpr (is_f64<T>()) {
        return (slot & 1u) ? u53(w.c, w.d) : u53(w.a, w.b);
    } else {
        const uint32_t q = slot & 3u;
        return u24(q == 0 ? w.a : q == 1 ? w.b : q == 2 ? w.c : w.d);
    }
}

// e- + Ar collision of the particle in `slot` (post-push state in memory),
// including the append record and the deposition of an ionisation pair.
// With `test`, the slot is a candidate that the particle loop's bound could
// not settle: the direct test of Algorithm 6 (P_coll of its fine table
// entry against its test uniform) is taken first, and the particle
// collides only if it passes.
template <typename T>
__device__ __forceinline__ void electron_collision(const DischargeDev &D, int slot, const RngKey &key, T idx_scale,
                                                   int cs_n, T inv_dx, int xcol,
                                                   unsigned int *sCnt, bool test, T ndt, T dt)
{
    using T2 = typename VecOf<T>::pair;
    T *X = reinterpret_cast<T *>(D.x[0]);
    T *VX = reinterpret_cast<T *>(D.vx[0]);
    T *VY = reinterpret_cast<T *>(D.vy[0]);
    T *VZ = reinterpret_cast<T *>(D.vz[0]);
    const T xn = X[slot];
    T vx = VX[slot], vy = VY[slot], vz = VZ[slot];
    const T v2 = sq3(vx, vy, vz);
    int k;
    if constexpr (is_f64<T>())
        k = cs_index(D.half_me * v2 / EDUPIC_QE, idx_scale, cs_n);
    else
        k = cs_index_f(madd(v2, idx_scale, 0.5f), cs_n);
    if (test) {
        const T sg = __ldg(reinterpret_cast<const T *>(D.cs_sig[0]) + k);
        const T speed = sqrt(v2);
        T pc;
        if constexpr (is_f64<T>())
            pc = p_coll(sg * ndt * speed * dt);
        else
            pc = p_coll(sg * ndt * speed);
        if (!(test_uniform<T, 0>(key, (uint32_t)slot) < pc)) return;
    }
    const T2 thr = reinterpret_cast<const T2 *>(D.cs_thr[0])[k];
    T u_proc, u_chi, u_eta, u_opal, vej[3];
    draw<T>(key, (uint32_t)slot, 0, 1, u_proc, u_chi);
    draw<T>(key, (uint32_t)slot, 0, 2, u_eta, u_opal);
    int sub;
    const int proc = collide_electron<T>(D, thr.x, thr.y, vx, vy, vz, u_proc, u_chi, u_eta, u_opal, vej, sub);
    VX[slot] = vx;
    VY[slot] = vy;
    VZ[slot] = vz;
    atomicAdd(sCnt + EDUPIC_C_COLL_E_ELA + proc, 1u);
    if (sub) atomicAdd(sCnt + EDUPIC_C_SUBTHRESHOLD, 1u);
    if (proc != 2) return;
    T n0, n1, n2, n3, z0, z1, z2, z3;
    draw<T>(key, (uint32_t)slot, 0, 3, n0, n1);
    draw<T>(key, (uint32_t)slot, 0, 4, n2, n3);
    box_muller(n0, n1, z0, z1);
    box_muller(n2, n3, z2, z3);
    const T sth = is_f64<T>() ? (T)D.sig_th : (T)D.sig_thf;
    const int pi = atomicAdd(&D.ctrl->products, 1);
    if (pi >= kEvents) {
        atomicOr(&D.ctrl->error, kErrProducts);
        return;
    }
    D.prod_parent[pi] = slot;
    reinterpret_cast<T *>(D.prod_x)[pi] = xn;
    reinterpret_cast<T *>(D.prod_ve[0])[pi] = vej[0];
    reinterpret_cast<T *>(D.prod_ve[1])[pi] = vej[1];
    reinterpret_cast<T *>(D.prod_ve[2])[pi] = vej[2];
    reinterpret_cast<T *>(D.prod_vi[0])[pi] = sth * z0;
    reinterpret_cast<T *>(D.prod_vi[1])[pi] = sth * z1;
    reinterpret_cast<T *>(D.prod_vi[2])[pi] = sth * z2;
    // the new pair joins the next densities at the parent's x
    T d0;
    const int pp = cell<T>(xn, inv_dx, D.ng, d0);
    const unsigned long long q2 = split_q2(d0 - (T)pp);
    // straight into the discharge's accumulators (products are rare), so the
    // block's shared counters take one deposit per particle pushed
    atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_e + pp), 4294967296ull - q2);
    atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_e + pp + 1), q2);
    atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_i + pp), 4294967296ull - q2);
    atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_i + pp + 1), q2);
    if (xcol >= 0) {
        // ionisation rate map: the event at the collision position
        atomicAdd(D.xt_ion + (size_t)pp * D.nxt + xcol, (double)((T)(pp + 1) - d0));
        atomicAdd(D.xt_ion + (size_t)(pp + 1) * D.nxt + xcol, (double)(d0 - (T)pp));
    }
}

// Thermal Ar partner of an ion (drawn before the collision probability).
template <typename T>
__device__ __forceinline__ void ion_partner(const DischargeDev &D, const RngKey &key, uint32_t slot, T &vax, T &vay,
                                            T &vaz)
{
    T a0, a1, a2, a3, za, zb, zc, zd;
    draw<T>(key, slot, 1, 1, a0, a1);
    draw<T>(key, slot, 1, 2, a2, a3);
    box_muller(a0, a1, za, zb);
    box_muller(a2, a3, zc, zd);
    const T sth = is_f64<T>() ? (T)D.sig_th : (T)D.sig_thf;
    vax = sth * za;
    vay = sth * zb;
    vaz = sth * zc;
}

template <typename T>
__device__ __forceinline__ int ion_index(const DischargeDev &D, T g_sqr, T idx_scale, int cs_n)
{
    if constexpr (is_f64<T>())
        return cs_index(D.half_mu_arar * g_sqr / EDUPIC_QE, idx_scale, cs_n);
    else
        return cs_index_f(madd(g_sqr, idx_scale, 0.5f), cs_n);
}

// Null-collision test of a particle picked by its test uniform u < P*
// (post-push velocity): the table index of its energy (e-) or of its relative
// energy with a thermal partner drawn now (Ar+, the same draws the collider
// makes), then u / P* < nu / nu*.  Called for the picked particles only.
template <typename T, int SP>
__device__ __noinline__ bool null_pick(const DischargeDev *Dp, const RngKey key, int slot, T vx, T vy, T vz, T u,
                                       T idx_scale, int cs_n, unsigned int *sCnt)
{
    const DischargeDev &D = *Dp;
    T q2;
    int k;
    if constexpr (SP == 0) {
        q2 = sq3(vx, vy, vz);
        if constexpr (is_f64<T>())
            k = cs_index(D.half_me * q2 / EDUPIC_QE, idx_scale, cs_n);
        else
            k = cs_index_f(madd(q2, idx_scale, 0.5f), cs_n);
    } else {
        T vax, vay, vaz;
        ion_partner<T>(D, key, (uint32_t)slot, vax, vay, vaz);
        const T gx = vx - vax, gy = vy - vay, gz = vz - vaz;
        q2 = sq3(gx, gy, gz);
        k = ion_index<T>(D, q2, idx_scale, cs_n);
    }
    return null_real<T, SP>(D, k, q2, u, sCnt);
}

// The direct collision test of Algorithm 6 for an Ar+ that the short cut
// could not settle (a few per cent): the thermal partner drawn before the
// probability; the table index of the relative energy; an exact coarse
// bound, then the fine entry.
template <typename T, int SP>
__device__ __forceinline__ bool direct_test_body(const DischargeDev *Dp, const RngKey key, int slot, T vx, T vy,
                                                 T vz, T v2, T u, T idx_scale, int cs_n, int cs_shift, const T *sC,
                                                 T ndt, T dt)
{
    const DischargeDev &D = *Dp;
    T q2 = v2;
    if constexpr (SP == 1) {
        T vax, vay, vaz;
        ion_partner<T>(D, key, (uint32_t)slot, vax, vay, vaz);
        q2 = sq3(vx - vax, vy - vay, vz - vaz);
    }
    int k;
    if constexpr (is_f64<T>())
        k = cs_index((SP == 0 ? D.half_me : D.half_mu_arar) * q2 / EDUPIC_QE, idx_scale, cs_n);
    else
        k = cs_index_f(madd(q2, idx_scale, 0.5f), cs_n);
    const T speed = sqrt(q2);
    T xu;
    if constexpr (is_f64<T>())
        xu = sC[k >> cs_shift] * ndt * speed * dt * 1.000001 + 1e-15;
    else
        xu = madd(sC[k >> cs_shift] * ndt * speed, 1.00001f, 1e-6f);
    if (!(u < xu)) return false;
    const T sg = __ldg(reinterpret_cast<const T *>(D.cs_sig[SP]) + k);
    T pc;
    if constexpr (is_f64<T>())
        pc = p_coll(sg * ndt * speed * dt);
    else
        pc = p_coll(sg * ndt * speed);
    return u < pc;
}

// Out of line: the partner draw (two Philox blocks, two Box-Muller pairs)
// in the unrolled particle loop overflowed the instruction cache (measured:
// 5 warps per issue stalled on instruction fetch in line, 0.5 out of line).
template <typename T, int SP>
__device__ __noinline__ bool direct_test_ool(const DischargeDev *Dp, const RngKey key, int slot, T vx, T vy, T vz,
                                             T v2, T u, T idx_scale, int cs_n, int cs_shift, const T *sC, T ndt,
                                             T dt)
{
    return direct_test_body<T, SP>(Dp, key, slot, vx, vy, vz, v2, u, idx_scale, cs_n, cs_shift, sC, ndt, dt);
}

// Ar+ + Ar collision of the ion in `slot` with its thermal partner.
template <typename T>
__device__ __forceinline__ void ion_collision(const DischargeDev &D, int slot, const RngKey &key, T idx_scale, int cs_n,
                                              unsigned int *sCnt)
{
    using T2 = typename VecOf<T>::pair;
    T *VX = reinterpret_cast<T *>(D.vx[1]);
    T *VY = reinterpret_cast<T *>(D.vy[1]);
    T *VZ = reinterpret_cast<T *>(D.vz[1]);
    T vx = VX[slot], vy = VY[slot], vz = VZ[slot];
    T vax, vay, vaz;
    ion_partner<T>(D, key, (uint32_t)slot, vax, vay, vaz);
    const T gx = vx - vax, gy = vy - vay, gz = vz - vaz;
    const int k = ion_index<T>(D, sq3(gx, gy, gz), idx_scale, cs_n);
    const T thr1 = reinterpret_cast<const T2 *>(D.cs_thr[1])[k].x;
    T u_proc, u_chi, u_eta, u_dummy;
    draw<T>(key, (uint32_t)slot, 1, 3, u_proc, u_chi);
    draw<T>(key, (uint32_t)slot, 1, 4, u_eta, u_dummy);
    const int proc = collide_ion<T>(D, thr1, vx, vy, vz, vax, vay, vaz, u_proc, u_chi, u_eta);
    VX[slot] = vx;
    VY[slot] = vy;
    VZ[slot] = vz;
    atomicAdd(sCnt + EDUPIC_C_COLL_I_ISO + proc, 1u);
}

// Particle that left the gap (Sec. 2.1.5), with the surface processes of
// Sec. 5.  An electron is first offered elastic reflection (block 5, R01 <
// eta of the electrode): the mirror image x -> -x (or 2L - x), if inside
// the gap, is returned and the caller continues with it and v_x reversed.
// Otherwise the particle is absorbed: its hole is recorded and counted, and
// for Ar+ the impact energy is binned into the IFED and an electron may be
// emitted (block 5, R01 < gamma of the electrode; blocks 6, 7: a
// half-Maxwellian velocity at the emission temperature pointing into the
// gap).  Emitted electrons start at the electrode, join the next electron
// densities here and the particle arrays when the step is finalized.
// Returns the mirror position, or -1 when the particle is absorbed.
template <typename T, int SP>
__device__ __noinline__ T absorbed(const DischargeDev *Dp, const RngKey key, int slot, T xn, T vx, T vy, T vz,
                                   int measure, unsigned int *sCnt)
{
    const DischargeDev &D = *Dp;
    const T L = is_f64<T>() ? (T)D.L : (T)D.Lf;
    const int side = xn < (T)0.0 ? 0 : (xn > L ? 1 : -1);
    if (SP == 0 && side >= 0 && D.refl_eta[side] > 0.0) {
        T u0, u1;
        draw<T>(key, (uint32_t)slot, 0, 5, u0, u1);
        const T eta = is_f64<T>() ? (T)D.refl_eta[side] : (T)D.refl_etaf[side];
        const T xr = side == 0 ? -xn : (T)2.0 * L - xn;
        if (u0 < eta && xr >= (T)0.0 && xr <= L) {
            atomicAdd(sCnt + EDUPIC_C_REFLECTED, 1u);
            return xr;
        }
    }
    if (side < 0)
        atomicOr(&D.ctrl->error, kErrNan);
    else
        atomicAdd(sCnt + (SP == 0 ? EDUPIC_C_ABS_E_POW : EDUPIC_C_ABS_I_POW) + side, 1u);
    const int h = atomicAdd(&D.ctrl->holes[SP], 1);
    if (h < kEvents)
        D.holes[SP][h] = slot;
    else
        atomicOr(&D.ctrl->error, kErrHoles);
    if (SP == 1 && measure && side >= 0) {
        const T v2 = vx * vx + vy * vy + vz * vz;
        int b;
        bool ok;
        if constexpr (is_f64<T>()) {
            const double en = D.half_mar * v2 / EDUPIC_QE;
            const double r = en / D.ifed_de;
            ok = r < (double)D.ifed_bins;
            b = ok ? (int)r : 0;
        } else {
            const float r = D.e_of_v2_if * v2 * D.inv_ifed_def;
            ok = r < (float)D.ifed_bins;
            b = ok ? (int)r : 0;
        }
        if (ok) atomicAdd((side == 0 ? D.ifed_pow : D.ifed_gnd) + b, 1ull);
    }
    if (SP == 1 && side >= 0 && D.see_gamma[side] > 0.0) {
        T u0, u1;
        draw<T>(key, (uint32_t)slot, 1, 5, u0, u1);
        const T gam = is_f64<T>() ? (T)D.see_gamma[side] : (T)D.see_gammaf[side];
        if (u0 < gam) {
            T a0, a1, b0, b1, za, zb, zc, zd;
            draw<T>(key, (uint32_t)slot, 1, 6, a0, a1);
            draw<T>(key, (uint32_t)slot, 1, 7, b0, b1);
            box_muller(a0, a1, za, zb);
            box_muller(b0, b1, zc, zd);
            const T sth = is_f64<T>() ? (T)D.see_sth : (T)D.see_sthf;
            const T xe = side == 0 ? (T)0.0 : L;
            atomicAdd(sCnt + EDUPIC_C_EMITTED_POW + side, 1u);
            const int ei = atomicAdd(&D.ctrl->emitted, 1);
            if (ei >= kEvents) {
                atomicOr(&D.ctrl->error, kErrProducts);
                return (T)-1.0;
            }
            D.emit_parent[ei] = slot;
            reinterpret_cast<T *>(D.emit_x)[ei] = xe;
            reinterpret_cast<T *>(D.emit_v[0])[ei] = (side == 0 ? sth : -sth) * fabs(za);
            reinterpret_cast<T *>(D.emit_v[1])[ei] = sth * zb;
            reinterpret_cast<T *>(D.emit_v[2])[ei] = sth * zc;
            T d0;
            const int pp = cell<T>(xe, is_f64<T>() ? (T)D.inv_dx : (T)D.inv_dxf, D.ng, d0);
            const unsigned long long q2 = split_q2(d0 - (T)pp);
            atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_e + pp), 4294967296ull - q2);
            atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_e + pp + 1), q2);
        }
    }
    return (T)-1.0;
}

// EEPF sample (Sec. 3.5): electrons in the centre 10% of the gap, energy of
// the time-centred velocity.
template <typename T>
__device__ __forceinline__ void eepf_sample(const DischargeDev *Dp, T vxc, T vy, T vz)
{
    const DischargeDev &D = *Dp;
    const T v2c = sq3(vxc, vy, vz);
    int b;
    bool ok;
    if constexpr (is_f64<T>()) {
        const double en = 0.5 * EDUPIC_ME * v2c / EDUPIC_QE;
        const double r = en / D.eepf_de;
        ok = r < (double)D.eepf_bins;
        b = ok ? (int)r : 0;
    } else {
        const float r = D.e_of_v2_ef * v2c * D.inv_eepf_def;
        ok = r < (float)D.eepf_bins;
        b = ok ? (int)r : 0;
    }
    // striped over kEepfStripes copies to spread the atomics; summed on read
    if (ok) atomicAdd(D.eepf + (blockIdx.x & (kEepfStripes - 1)) * D.eepf_bins + b, 1ull);
}

// ---------------------------------------------------------------- particle kernel
// Launch shapes (push_shape_of): the xt-accumulating variant has a shape of
// its own, whose fourth FP32 stage's room holds the xt sums.
template <typename T>
__host__ __device__ constexpr PushShape push_shape(int s)
{
    return push_shape_of(is_f64<T>(), s);
}
template <typename T>
__host__ __device__ constexpr PushShape push_shape_xt()
{
    return PushShape{256, 3, 2};
}
template <typename T, bool XT, int SH>
__host__ __device__ constexpr PushShape shape_of()
{
    return XT ? push_shape_xt<T>() : push_shape<T>(SH);
}

// Dynamic shared memory: [tile ring: stages x 4 arrays x TILE T][bound
// table: kCoarse T (e-: the threshold of each v^2 bucket; Ar+: the coarse
// sigma_max)][field: ng_max T2 (FP64: E_p, E_p+1; FP32: E_p, E_p+1 - E_p)]
// [deposition: 3 x ng_max u32][tile prefix: nd+1 int][xt variant, from the
// next 16-byte boundary: sum w v_c,x and sum w eps_c, ng_max T each].
template <typename T, bool XT, int SH>
__host__ __device__ constexpr size_t push_smem_bytes(int nd, int ng_max, int eepf_max)
{
    return (size_t)shape_of<T, XT, SH>().stages * 4 * shape_of<T, XT, SH>().threads * VecOf<T>::n * sizeof(T) +
           (size_t)kCoarse * sizeof(T) + (size_t)ng_max * 2 * sizeof(T) + (size_t)ng_max * 12 + (size_t)(nd + 1) * 4 +
           (XT ? 16 + (size_t)ng_max * 2 * sizeof(T) : 0) + 0 * (size_t)eepf_max;
}

// NC: the variant that also runs the null-collision method for the
// discharges that ask for it (launched only when one does; the direct-test
// variant carries none of its code).
// XT: the variant that also accumulates the xt diagnostics of the measured
// steps (launched only for measured steps of a simulation that keeps them).
// AGG: the variant for discharges that keep their particles in cell order
// (the periodic sort), whose deposits go through warp-level reductions
// (launched only when one does: the others carry none of its code).
template <typename T, int SP, bool NC, bool XT, int SH, bool AGG = false>
__global__ void __launch_bounds__(shape_of<T, XT, SH>().threads, shape_of<T, XT, SH>().min_blocks)
    k_push(const DischargeDev *__restrict__ DD, int nd, int ng_max, int eepf_max, int measure)
{
    using V = typename VecOf<T>::type;
    using T2 = typename VecOf<T>::pair;
    constexpr int VEC = VecOf<T>::n;  // slots per thread: one Philox test block
    constexpr int NTHR = shape_of<T, XT, SH>().threads;
    constexpr int TILE = NTHR * VEC;
    constexpr int S = shape_of<T, XT, SH>().stages;
    constexpr int kWarps = NTHR / 32;
    static_assert(TILE <= 1024 && 1024 % TILE == 0, "tiles stay inside the particle arrays' padding");
    static_assert(kWarpQueue >= 2 * 32 * VEC, "a warp queue takes at least two tiles of colliders");
    extern __shared__ __align__(128) unsigned char smem[];
    T *sRing = reinterpret_cast<T *>(smem);  // [stage][array x, vx, vy, vz][TILE]
    T *sC = sRing + S * 4 * TILE;
    T2 *sE2 = reinterpret_cast<T2 *>(sC + kCoarse);
    DepAcc acc;
    acc.cnt = reinterpret_cast<unsigned int *>(sE2 + ng_max);
    acc.lo = acc.cnt + ng_max;
    acc.hi = acc.lo + ng_max;
    acc.s_cnt = (uint32_t)__cvta_generic_to_shared(acc.cnt);
    acc.s_lo = (uint32_t)__cvta_generic_to_shared(acc.lo);
    acc.s_hi = (uint32_t)__cvta_generic_to_shared(acc.hi);
    int *sPre = reinterpret_cast<int *>(acc.hi + ng_max);
    // xt variant: sum w v_c,x and sum w eps_c of the block, per grid point, on a
    // 16-byte boundary after the prefix (whose end is 4-byte aligned only)
    T *sXv = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(sPre + nd + 1) + 15) & ~(uintptr_t)15);
    T *sXe = sXv + ng_max;
    (void)eepf_max;
    __shared__ unsigned int sCnt[EDUPIC_N_COUNTERS];
    __shared__ int sW[33];
    __shared__ int sQueue[kWarps][kWarpQueue];  // colliders queued by each warp
    __shared__ int sQn[kWarps];
    __shared__ uint4 sRK[5];  // Philox round keys of the current discharge (philox_rk)
    __shared__ DischargeDev sD;  // descriptor of the discharge being processed

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // set-up data that does not depend on the preceding kernel, fetched
    // before waiting for it: the coarse table (shared by all discharges) and
    // the descriptor of discharge 0
    if constexpr (SP == 1) {
        const float4 *cm = reinterpret_cast<const float4 *>(DD[0].cs_max[SP]);
        float4 *dst = reinterpret_cast<float4 *>(sC);
        for (int j = tid; j < (int)(kCoarse * sizeof(T) / 16); j += blockDim.x) dst[j] = cm[j];
    }
    {
        const int *src = reinterpret_cast<const int *>(DD);
        int *dd = reinterpret_cast<int *>(&sD);
        for (int i = tid; i < (int)(sizeof(DischargeDev) / 4); i += blockDim.x) dd[i] = src[i];
    }
    if (tid < kWarps) sQn[tid] = 0;
    if (tid < EDUPIC_N_COUNTERS) sCnt[tid] = 0;
    __syncthreads();
    const int cs_shift = sD.cs_shift[SP];
    const Ctrl *ctrls = sD.ctrl;  // the counts of all discharges are one packed array
    int staged = 0;
    pdl_wait();
    pdl_launch_next();
    // tiles per discharge -> prefix over discharges (every block computes it)
    {
        int running = 0;
        for (int base = 0; base < nd; base += blockDim.x) {
            const int d = base + tid;
            int cnt = 0;
            if (d < nd && DD[d].active && ctrls[d].step < DD[d].stop_step)
                cnt = (int)((ctrls[d].n[SP] + TILE - 1) / TILE);
            int tot;
            const int ex = group_excl_scan(cnt, sW, tot, tid, blockDim.x, 1);
            if (d < nd) sPre[d] = running + ex;
            running += tot;
        }
        if (tid == 0) sPre[nd] = running;
    }
    __syncthreads();
    const int total = sPre[nd];
    const int t0 = (int)((long long)blockIdx.x * total / gridDim.x);
    const int t1 = (int)((long long)(blockIdx.x + 1) * total / gridDim.x);
    if (t0 >= t1) return;

    const DischargeDev *D = &sD;
    int cur = -1;
    int n = 0, cs_n = 0, ng = 0;
    uint32_t s_lo = 0, s_hi = 0, k0 = 0, k1 = 0;
    T L = 0, inv_dx = 0, dt = 0, factor = 0, ndt = 0, idx_scale = 0, lo = 0, hi = 0;
    const T *sig = nullptr;
    T *X = nullptr, *VX = nullptr, *VY = nullptr, *VZ = nullptr;
    bool eepf_on = false;
    bool nullc = false;  // null-collision method for the current discharge
    T pstar = 0;         // its P*
    T v2top = 0, gcap = 0;     // bound of the Ar+ direct test
    const T *pm = nullptr;    // prefix maxima of sigma_tot * v (Ar+ bound)
    float eepf_k = 0.f, eepf_nbf = 0.f;
    unsigned long long *eepf_row = nullptr;
    int xcol = -1;       // xt time bin of this step for the current discharge (-1: none)
    T e_of_v2 = 0;       // energy in eV of v^2 (xt variant)
    int lv_base = 0, lv_n = 1;  // electrons: v^2 buckets of the bound table

    // execute the collisions queued by this warp (the 32 lanes of the warp;
    // the particles were stored by lanes of the same warp, ordered by the
    // warp barrier)
    auto drain = [&]() {
        __syncwarp();
        const int qn = sQn[warp];
        if (qn == 0) return;  // uniform across the warp: read after the warp barrier
        const RngKey key{s_lo, s_hi, k0, k1};
        for (int i = lane; i < qn; i += 32) {
            if (SP == 0)
                electron_collision<T>(*D, sQueue[warp][i], key, idx_scale, cs_n, inv_dx, XT ? xcol : -1, sCnt,
                                      !(NC && nullc), ndt, dt);
            else
                ion_collision<T>(*D, sQueue[warp][i], key, idx_scale, cs_n, sCnt);
        }
        __syncwarp();
        if (lane == 0) sQn[warp] = 0;
        __syncwarp();
    };

    // add the block's deposition into the discharge's accumulator (and clear it)
    auto flush_dep = [&](bool clear) {
        __syncthreads();
        long long *accq = SP == 0 ? D->acc_e : D->acc_i;
        for (int p = tid; p < ng; p += blockDim.x) {
            const unsigned long long q = (dep_cnt(acc, p) << 32) - dep_sum(acc, p) +
                                         (p > 0 ? dep_sum(acc, p - 1) : 0ull);
            if (q) atomicAdd(reinterpret_cast<unsigned long long *>(accq + p), q);
            if constexpr (XT) {
                if (xcol >= 0) {
                    const size_t j = (size_t)p * D->nxt + xcol;
                    if (sXv[p] != (T)0) atomicAdd(D->xt_v[SP] + j, (double)sXv[p]);
                    if (sXe[p] != (T)0) atomicAdd(D->xt_en[SP] + j, (double)sXe[p]);
                }
            }
        }
        if (!clear) return;
        __syncthreads();
        for (int p = tid; p < ng; p += blockDim.x) {
            acc.cnt[p] = acc.lo[p] = acc.hi[p] = 0u;
            if constexpr (XT) sXv[p] = sXe[p] = (T)0;
        }
        __syncthreads();
    };

    double pw_acc = 0.0;  // E_x (v_old + v_new) of this thread's measured pushes (current discharge)
    int picks = 0;        // null-collision picks of this thread (current discharge)

    auto flush = [&](bool last) {
        drain();
        flush_dep(!last);
        if (measure) {
            // power absorption: warp sums, one add per warp
            double v = pw_acc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0 && v != 0.0) atomicAdd(D->power + SP, v);
            pw_acc = 0.0;
        }
        if constexpr (NC) {
            // null-collision picks: warp sums, one add per warp
            int pk = picks;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pk += __shfl_down_sync(0xffffffffu, pk, o);
            if (lane == 0 && pk) atomicAdd(D->ctrl->counters + EDUPIC_C_NULL_TESTED, (unsigned long long)pk);
            picks = 0;
        }
        if (tid < EDUPIC_N_COUNTERS) {
            const unsigned int c = sCnt[tid];
            if (c) atomicAdd(D->ctrl->counters + tid, (unsigned long long)c);
            sCnt[tid] = 0;
        }
        if (!last) __syncthreads();
    };

    int since_flush = 0;
    T xa[VEC], vxa[VEC], vya[VEC], vza[VEC];  // particles of this thread in the current tile

    // Tile ring: every thread copies its own VEC particles (16 bytes per array;
    // whole tiles stay inside the padded capacity) of tile `pt` into stage
    // `st` and reads back only those, so no thread
    // waits for another; each tile is one commit group, S - 1 tiles ahead.
    // The discharge of the tile being fetched (pcur) is cached with its tile
    // range and this thread's source address in its x array; v_x, v_y, v_z
    // follow at equal strides.
    int pt = t0, pcur = -1, la_base = 0, la_end = 0;
    const char *la_src = nullptr;
    long long la_stride = 0;
    const uint32_t ring_me = (uint32_t)__cvta_generic_to_shared(sRing + tid * VEC);
    auto issue = [&](int st) {
        if (pt < t1) {
            if (pt >= la_end) {
                do {
                    ++pcur;
                } while (pt >= sPre[pcur + 1]);
                la_base = sPre[pcur];
                la_end = sPre[pcur + 1];
                const DischargeDev *Dq = DD + pcur;
                la_src = reinterpret_cast<const char *>(__ldg(reinterpret_cast<const unsigned long long *>(&Dq->x[SP]))) +
                         (size_t)tid * VEC * sizeof(T);
                la_stride = __ldg(&Dq->pstride[SP]);
            }
            const char *src = la_src + (size_t)(pt - la_base) * (TILE * sizeof(T));
            const uint32_t dst = ring_me + (uint32_t)(st * 4 * TILE * (int)sizeof(T));
            cp_async16(dst, src);
            cp_async16(dst + TILE * sizeof(T), src + la_stride);
            cp_async16(dst + 2 * TILE * sizeof(T), src + 2 * la_stride);
            cp_async16(dst + 3 * TILE * sizeof(T), src + 3 * la_stride);
            ++pt;
        }
        cp_async_commit();  // one group per tile, empty past the block's last tile
    };
#pragma unroll
    for (int k = 0; k < S - 1; ++k) issue(k);

    int cur_base = 0, cur_end = 0;  // tile range of the current discharge
    for (int t = t0, st = 0; t < t1; ++t, st = st + 1 == S ? 0 : st + 1) {
        if (t >= cur_end) {
            if (cur >= 0) flush(false);
            ++cur;
            while (sPre[cur + 1] <= t) ++cur;
            cur_base = sPre[cur];
            cur_end = sPre[cur + 1];
            if (cur != staged) {
                const int *src = reinterpret_cast<const int *>(DD + cur);
                int *dd = reinterpret_cast<int *>(&sD);
                for (int i = tid; i < (int)(sizeof(DischargeDev) / 4); i += blockDim.x) dd[i] = src[i];
                __syncthreads();
                staged = cur;
            }
            n = (int)ctrls[cur].n[SP];
            const unsigned long long s = (unsigned long long)ctrls[cur].step;
            s_lo = (uint32_t)s;
            s_hi = (uint32_t)(s >> 32);
            k0 = (uint32_t)D->seed;
            k1 = (uint32_t)(D->seed >> 32);
            ng = D->ng;
            if constexpr (is_f64<T>()) {
                L = D->L;
                inv_dx = D->inv_dx;
                dt = SP == 0 ? D->dt_e : D->dt_i;
                factor = SP == 0 ? D->factor_e : D->factor_i;
                ndt = D->n_gas;
                idx_scale = SP == 0 ? D->cs_de_e : D->cs_de_i;
                lo = D->eepf_lo;
                hi = D->eepf_hi;
            } else {
                L = D->Lf;
                inv_dx = D->inv_dxf;
                dt = SP == 0 ? D->dt_ef : D->dt_if;
                factor = SP == 0 ? D->factor_ef : D->factor_if;
                ndt = SP == 0 ? D->ndt_ef : D->ndt_if;
                idx_scale = SP == 0 ? D->e_idx_ef : D->g_idx_if;
                lo = D->eepf_lof;
                hi = D->eepf_hif;
            }
            sig = reinterpret_cast<const T *>(D->cs_sig[SP]);
            X = reinterpret_cast<T *>(D->x[SP]);
            VX = reinterpret_cast<T *>(D->vx[SP]);
            VY = reinterpret_cast<T *>(D->vy[SP]);
            VZ = reinterpret_cast<T *>(D->vz[SP]);
            cs_n = SP == 0 ? D->cs_n_e : D->cs_n_i;
            eepf_on = SP == 0 && measure;
            if (!eepf_on) lo = (T)INFINITY;  // an empty sampling window: no position is at or above it
            if constexpr (NC) {
                nullc = ((D->null_coll >> SP) & 1) != 0;
                pstar = is_f64<T>() ? (T)D->p_star[SP] : (T)D->p_starf[SP];
            }
            eepf_k = D->e_of_v2_ef * D->inv_eepf_def;
            eepf_nbf = (float)D->eepf_bins;
            eepf_row = D->eepf + (blockIdx.x & (kEepfStripes - 1)) * D->eepf_bins;
            pm = reinterpret_cast<const T *>(D->cs_pm[SP]);
            if constexpr (is_f64<T>()) {
                v2top = D->v2top[SP];
                gcap = D->gcap;
            } else {
                v2top = D->v2topf[SP];
                gcap = D->gcapf;
            }
            if constexpr (XT) {
                xcol = (measure && D->nxt > 0) ? (int)((long long)(s % (unsigned long long)D->nt) / D->nbin) : -1;
                if constexpr (is_f64<T>())
                    e_of_v2 = (SP == 0 ? D->half_me : D->half_mar) / EDUPIC_QE;
                else
                    e_of_v2 = SP == 0 ? D->e_of_v2_ef : D->e_of_v2_if;
            }
            if (tid < 5) {
                // round keys of the test draws: k0 + r 0x9E3779B9, k1 + r 0xBB67AE85 (rounds 2 tid, 2 tid + 1)
                const uint32_t r = 2u * (uint32_t)tid;
                sRK[tid] = make_uint4(k0 + r * 0x9E3779B9u, k1 + r * 0xBB67AE85u, k0 + (r + 1u) * 0x9E3779B9u,
                                      k1 + (r + 1u) * 0xBB67AE85u);
            }
            if constexpr (SP == 0) {
                // electrons' collision bound per v^2 bucket: n dt max(sigma_tot v)
                // over the bucket (the table holds max sigma_tot v, rounded up),
                // widened past the rounding of the test's own arithmetic
                lv_base = D->lv_base;
                lv_n = D->lv_n;
                const T *mt = reinterpret_cast<const T *>(D->cs_max[0]);
                for (int j = tid; j < lv_n; j += blockDim.x) {
                    if constexpr (is_f64<T>()) {
                        sC[j] = mt[j] * ndt * dt * 1.000001 + 1e-15;
                    } else {
                        // FP32: the bound B as the integer threshold of the test
                        // word, u = (w >> 8) 2^-24 < B  <=>  (w >> 8) < ceil(B 2^24)
                        const float b = madd(mt[j] * ndt, 1.00001f, 1e-6f) * 16777216.0f;
                        reinterpret_cast<uint32_t *>(sC)[j] = b >= 16777216.0f ? 16777216u : (uint32_t)ceilf(b);
                    }
                }
            }
            const T *ef = reinterpret_cast<const T *>(D->ef_t);
            for (int p = tid; p < ng; p += blockDim.x) {
                // FP64: (E_p, E_p+1); FP32: (E_p, E_p+1 - E_p), the slope the
                // linear weights take (the same FP32 difference the push formed)
                const T e1 = p + 1 < ng ? ef[p + 1] : (T)0;
                sE2[p] = is_f64<T>() ? T2{ef[p], e1} : T2{ef[p], e1 - ef[p]};
                acc.cnt[p] = acc.lo[p] = acc.hi[p] = 0u;
                if constexpr (XT) sXv[p] = sXe[p] = (T)0;
            }
            since_flush = 0;
            __syncthreads();
        }
        const int tbase = (t - cur_base) * TILE;
        if (tid == 0) atomicAdd(sCnt + (SP == 0 ? EDUPIC_C_PUSH_E : EDUPIC_C_PUSH_I), (unsigned)min(TILE, n - tbase));
        const int base = tbase + tid * VEC;
        if (since_flush >= kDepFlush) {
            flush_dep(true);
            since_flush = 0;
        }
        since_flush += TILE;
        // a tile adds at most 32 * VEC colliders to this warp's queue
        if (sQn[warp] > kWarpQueue - 32 * VEC) drain();
        // the tile S - 1 ahead into the stage this thread read in the previous
        // iteration; then this tile's own copies (allowing S - 1 newer groups)
        issue(st ? st - 1 : S - 1);
        cp_async_wait<S - 1>();
        {
            const T *rs = sRing + (size_t)st * 4 * TILE + tid * VEC;
            unpack(*reinterpret_cast<const V *>(rs), xa);
            unpack(*reinterpret_cast<const V *>(rs + TILE), vxa);
            unpack(*reinterpret_cast<const V *>(rs + 2 * TILE), vya);
            unpack(*reinterpret_cast<const V *>(rs + 3 * TILE), vza);
        }
        // lanes with particles in this tile (every lane of the warp reaches this ballot)
        const unsigned int live_lanes = __ballot_sync(0xffffffffu, base < n);
        if (base >= n) continue;

        // collision-test draw (one Philox block per thread, Sec. 3.3): it
        // depends on the slots only, and its arithmetic interleaves with the
        // particles' own below.  tw: the raw words (FP32: u = (word >> 8) 2^-24)
        T ut[VEC];
        uint32_t tw[4];
        {
            const Words w = philox_rk((uint32_t)base / VEC, s_lo, s_hi, (uint32_t)SP << 8, sRK);
            tw[0] = w.a;
            tw[1] = w.b;
            tw[2] = w.c;
            tw[3] = w.d;
            if constexpr (is_f64<T>()) {
                uniforms(w, ut[0], ut[1]);
            } else {
                ut[0] = u24(w.a);
                ut[1] = u24(w.b);
                ut[2] = u24(w.c);
                ut[3] = u24(w.d);
            }
        }
        // phase 1: gather (Sec. 2.1.3), leapfrog push (Sec. 2.1.4), absorption
        // test (Sec. 2.1.5), and the first part of the collision test
        // (Algorithm 6): the particle's table entry and the bound that settles
        // most particles without it.  With x = n sigma_tot v dt, P_coll =
        // 1 - exp(-x) <= x, and the coarse maximum of sigma_tot bounds x from
        // above: R01 at or above that bound (plus a rounding margin) decides
        // "no collision".  The fine entry of the particles below it (and of
        // the null-collision picks) is fetched here, predicated, and used
        // after the deposition.
        bool in[VEC];
        bool cand[VEC];  // a candidate for a collision: the full test follows
        T sgp[VEC];      // e-: sigma_tot of the fine entry (candidates); Ar+: the bound's table value
        bool far[VEC];   // Ar+: relative speed bound past the table (always a candidate)
        T pw = (T)0;  // E_x (v_old + v_new) of the measured pushes of this tile
        // FP32: two particles per step of the loop through paired FP32
        // instructions (each lane rounds as the scalar operation); their
        // measured E_x (v_old + v_new) summed per lane
        constexpr int PR = is_f64<T>() ? 1 : 2;
        float2 pw2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int h = 0; h < VEC; h += PR) {
            T c0v[PR], exv[PR], vxnv[PR], xnv[PR], w2v[PR], rv[PR];
            int pv[PR];
            if constexpr (PR == 2) {
                const float2 xp = make_float2(xa[h], xa[h + 1]);
                const float2 vxp = make_float2(vxa[h], vxa[h + 1]);
                const float2 vyp = make_float2(vya[h], vya[h + 1]);
                const float2 vzp = make_float2(vza[h], vza[h + 1]);
                const float2 c0 = f2_mul(xp, make_float2(inv_dx, inv_dx));
                pv[0] = (int)min((unsigned)(int)c0.x, (unsigned)(ng - 2));
                pv[1] = (int)min((unsigned)(int)c0.y, (unsigned)(ng - 2));
                const T2 ep0 = sE2[pv[0]], ep1 = sE2[pv[1]];
                // c0 - p (one rounding, as the subtraction), then the linear weights
                const float2 fr = f2_fma(make_float2((float)pv[0], (float)pv[1]), make_float2(-1.0f, -1.0f), c0);
                const float2 ex = make_float2(madd(fr.x, ep0.y, ep0.x), madd(fr.y, ep1.y, ep1.x));
                // electrons: -e_x factor is e_x (-factor), the same product
                const float fs = SP == 0 ? -factor : factor;
                const float2 vxn = f2_fma(ex, make_float2(fs, fs), vxp);
                const float2 sv = f2_add(vxp, vxn);
                if (measure) {
                    const float2 t = f2_fma(ex, sv, pw2);
                    pw2.x = base + h < n ? t.x : pw2.x;
                    pw2.y = base + h + 1 < n ? t.y : pw2.y;
                }
                if constexpr (SP == 0) {
                    const float2 vxc = f2_mul(make_float2(0.5f, 0.5f), sv);
                    const float2 r = f2_mul(make_float2(eepf_k, eepf_k), f2_sq3(vxc, vyp, vzp));
                    rv[0] = r.x;
                    rv[1] = r.y;
                }
                const float2 xn = f2_fma(vxn, make_float2(dt, dt), xp);
                const float2 w2 = f2_sq3(vxn, vyp, vzp);
                c0v[0] = c0.x;
                c0v[1] = c0.y;
                exv[0] = ex.x;
                exv[1] = ex.y;
                vxnv[0] = vxn.x;
                vxnv[1] = vxn.y;
                xnv[0] = xn.x;
                xnv[1] = xn.y;
                w2v[0] = w2.x;
                w2v[1] = w2.y;
            } else {
                const T x = xa[h], vx = vxa[h];
                T c0;
                const int p = cell<T>(x, inv_dx, ng, c0);
                const T2 ep = sE2[p];
                const T c1 = (T)(p + 1) - c0, c2 = c0 - (T)p;
                const T e_x = c1 * ep.x + c2 * ep.y;
                const T vxn = SP == 0 ? madd(-e_x, factor, vx) : madd(e_x, factor, vx);
                if (measure && base + h < n) pw = madd(e_x, vx + vxn, pw);
                c0v[0] = c0;
                pv[0] = p;
                exv[0] = e_x;
                vxnv[0] = vxn;
                xnv[0] = madd(vxn, dt, x);
                w2v[0] = sq3(vxn, vya[h], vza[h]);
                rv[0] = (T)0;
            }
#pragma unroll
        for (int q = 0; q < PR; ++q) {
            const int e = h + q;
            const bool live = base + e < n;
            const T x = xa[e], vx = vxa[e];
            const T c0 = c0v[q], vxn = vxnv[q];
            const int p = pv[q];
            (void)exv;
            (void)vx;
            if constexpr (SP == 0 && !is_f64<T>()) {
                // EEPF sample (Sec. 3.5): every lane forms the bin and only the
                // atomic is predicated (a tenth of the electrons sample, so a
                // branch would be taken by some lane of almost every warp)
                // (the window is empty when not measuring; the bin's address is
                // formed by every lane and used only by those that sample)
                const bool take = live && x >= lo && x <= hi;
                const float r = rv[q];  // eepf_k sq3(v_c) of the time-centred velocity
                const bool okb = take && r < eepf_nbf;
                red_add1_global_if(eepf_row + (int)r, okb);
            } else if (SP == 0 && eepf_on && live && x >= lo && x <= hi) {
                eepf_sample<T>(D, (T)0.5 * (vx + vxn), vya[e], vza[e]);
            }
            if constexpr (XT) {
                // xt sums at x(t) with the time-centred velocity, weighted like the deposition
                if (xcol >= 0 && live) {
                    const T vc = (T)0.5 * (vx + vxn);
                    const T en = e_of_v2 * (vc * vc + vya[e] * vya[e] + vza[e] * vza[e]);
                    const T w1 = (T)(p + 1) - c0, w2 = c0 - (T)p;
                    atomicAdd(sXv + p, w1 * vc);
                    atomicAdd(sXv + p + 1, w2 * vc);
                    atomicAdd(sXe + p, w1 * en);
                    atomicAdd(sXe + p + 1, w2 * en);
                }
            }
            const T xn = xnv[q];
            // slots past the count (the last tile's padding) are pushed too and
            // written back to the padding, which holds no particle
            xa[e] = xn;
            vxa[e] = vxn;
            in[e] = live && (xn >= (T)0.0) && (xn <= L);
            // own squared speed after the push
            const T w2 = w2v[q];
            far[e] = false;
            if constexpr (SP == 0) {
                if (NC && nullc) {
                    // the null-collision pick, tested in place below with its fine entry
                    int k;
                    if constexpr (is_f64<T>())
                        k = cs_index(D->half_me * w2 / EDUPIC_QE, idx_scale, cs_n);
                    else
                        k = cs_index_f(madd(w2, idx_scale, 0.5f), cs_n);
                    cand[e] = live && ut[e] < pstar;
                    sgp[e] = ldg_if(sig + k, cand[e]);
                } else {
                    // the bound of the particle's v^2 bucket; candidates are
                    // tested against their fine entry in the collider
                    const int j = lv_bucket(w2, lv_base, lv_n);
                    if constexpr (is_f64<T>())
                        cand[e] = live && ut[e] < sC[j];
                    else
                        cand[e] = live && (tw[e] >> 8) < reinterpret_cast<const uint32_t *>(sC)[j];
                    sgp[e] = (T)0;
                }
            } else {
                // Ar+: the relative speed to any partner the generator can draw
                // is at most gm = |v| + gcap, so P_coll <= n dt max(sigma_tot v)
                // over the entries up to gm's (the prefix maximum); its table
                // value is fetched here and compared below
                const T gm = (sqrt(w2) + gcap) * (T)(1.0 + 1e-6);
                const T gm2 = gm * gm;
                far[e] = gm2 > v2top;  // past the table: no bound
                int k;
                if constexpr (is_f64<T>())
                    k = cs_index(D->half_mu_arar * gm2 / EDUPIC_QE, idx_scale, cs_n);
                else
                    k = cs_index_f(madd(gm2, idx_scale, 0.5f), cs_n);
                cand[e] = live;
                sgp[e] = ldg_if(pm + (k >> cs_shift), live && !far[e] && !(NC && nullc));
            }
        }
        }
        if (measure) pw_acc += (double)pw + (double)(pw2.x + pw2.y);
        // deposition of the new position for the next step (Sec. 2.1.1) of the
        // particles that stay in the gap (a reflected electron deposits below);
        // gathered below when the discharge keeps its particles in cell order
        int dcell[VEC];                // cell of each deposit (-1: none)
        unsigned long long dq2[VEC];  // its fixed-point weight of point cell + 1
#pragma unroll
        for (int h = 0; h < VEC; h += PR) {
            int ppv[PR];
            unsigned long long q2v[PR];
            if constexpr (PR == 2) {
                // the cell and weight of cell (x) and split_q2, two lanes per instruction
                const float2 c0 = f2_mul(make_float2(xa[h], xa[h + 1]), make_float2(inv_dx, inv_dx));
                ppv[0] = (int)min((unsigned)(int)c0.x, (unsigned)(ng - 2));
                ppv[1] = (int)min((unsigned)(int)c0.y, (unsigned)(ng - 2));
                const float2 c2 =
                    f2_fma(make_float2((float)ppv[0], (float)ppv[1]), make_float2(-1.0f, -1.0f), c0);
                const float2 sc = f2_mul(c2, make_float2(4294967296.0f, 4294967296.0f));
                q2v[0] = c2.x < 1.0f ? (unsigned long long)__float2uint_rn(sc.x) : 4294967296ull;
                q2v[1] = c2.y < 1.0f ? (unsigned long long)__float2uint_rn(sc.y) : 4294967296ull;
            } else {
                T d0;
                ppv[0] = cell<T>(xa[h], inv_dx, ng, d0);
                q2v[0] = split_q2(d0 - (T)ppv[0]);
            }
#pragma unroll
            for (int q = 0; q < PR; ++q) {
                const int e = h + q;
                if constexpr (AGG) {
                    dcell[e] = in[e] ? ppv[q] : -1;
                    dq2[e] = q2v[q];
                } else {
                    dep_add_if(acc, ppv[q], q2v[q], in[e]);
                }
            }
        }
        if constexpr (SP == 1) {
            // Ar+: the bound decides (null-collision method: the pick)
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                if (NC && nullc) {
                    cand[e] = cand[e] && ut[e] < pstar;
                } else {
                    T xb;
                    if constexpr (is_f64<T>())
                        xb = sgp[e] * ndt * dt * 1.000001 + 1e-15;
                    else
                        xb = madd(sgp[e] * ndt, 1.00001f, 1e-6f);
                    cand[e] = cand[e] && (far[e] || ut[e] < xb);
                }
            }
        }
        // the rare part, per lane: particles that left the gap (absorption,
        // reflection, emission) and the full collision test of the candidates;
        // colliding slots are queued (executed after the stores below)
        bool rare = false;
#pragma unroll
        for (int e = 0; e < VEC; ++e) rare = rare || cand[e] || (base + e < n && !in[e]);
        if (rare) {
            const RngKey key{s_lo, s_hi, k0, k1};
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int slot = base + e;
                bool go = cand[e];
                if (slot < n && !in[e]) {
                    const T xr = absorbed<T, SP>(D, key, slot, xa[e], vxa[e], vya[e], vza[e], measure, sCnt);
                    if (SP == 1 || xr < (T)0.0) {
                        go = false;
                    } else {
                        // reflected electron: continues in the gap (v^2 and the
                        // table index are unchanged) and deposits at its mirror image
                        xa[e] = xr;
                        vxa[e] = -vxa[e];
                        T d0;
                        const int pp = cell<T>(xr, inv_dx, ng, d0);
                        const unsigned long long q2 = split_q2(d0 - (T)pp);
                        if constexpr (AGG) {
                            dcell[e] = pp;
                            dq2[e] = q2;
                        } else {
                            dep_add(acc, pp, q2);
                        }
                    }
                }
                if (!go) continue;
                bool real;
                if constexpr (SP == 0) {
                    if (NC && nullc) {
                        ++picks;
                        real = null_real_sg<T, 0>(*D, sgp[e], sq3(vxa[e], vya[e], vza[e]), ut[e], sCnt);
                    } else {
                        real = true;  // a candidate: the collider takes the direct test
                    }
                } else {
                    if (NC && nullc) {
                        ++picks;
                        real = null_pick<T, SP>(D, key, slot, vxa[e], vya[e], vza[e], ut[e], idx_scale, cs_n, sCnt);
                    } else {
                        real = direct_test_ool<T, SP>(D, key, slot, vxa[e], vya[e], vza[e],
                                                      sq3(vxa[e], vya[e], vza[e]), ut[e], idx_scale, cs_n,
                                                      cs_shift, sC, ndt, dt);
                    }
                }
                if (real) sQueue[warp][atomicAdd(sQn + warp, 1)] = slot;
            }
        }
        // Deposition through warp-level reductions for a discharge that
        // keeps its particles in cell order (the periodic sort), whose
        // neighbouring slots share cells: all 32 x VEC deposits of the warp
        // in one cell -> one set of shared atomics for the warp; a thread's
        // VEC deposits in one cell -> one set for the thread; otherwise one
        // set per deposit.  The sums are the same integers in every case.
        if constexpr (AGG) {
            bool same = dcell[0] >= 0;
#pragma unroll
            for (int e = 1; e < VEC; ++e) same = same && dcell[e] == dcell[0];
            // the warp path only with all 32 lanes here (a warp-uniform branch)
            int c0w = -1;
            bool warp_same = false;
            if (live_lanes == 0xffffffffu) {
                c0w = __shfl_sync(0xffffffffu, dcell[0], 0);
                warp_same = __all_sync(0xffffffffu, same && dcell[0] == c0w);
            }
            if (warp_same) {
                unsigned int lo = 0u, hi = 0u;
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    lo += (unsigned int)(dq2[e] & 0xFFFFull);
                    hi += (unsigned int)(dq2[e] >> 16);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lo += __shfl_xor_sync(0xffffffffu, lo, o);
                    hi += __shfl_xor_sync(0xffffffffu, hi, o);
                }
                if (lane == 0) {
                    atomicAdd(acc.cnt + c0w, 32u * VEC);
                    atomicAdd(acc.lo + c0w, lo);
                    atomicAdd(acc.hi + c0w, hi);
                }
            } else if (same) {
                unsigned int lo = 0u, hi = 0u;
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    lo += (unsigned int)(dq2[e] & 0xFFFFull);
                    hi += (unsigned int)(dq2[e] >> 16);
                }
                atomicAdd(acc.cnt + dcell[0], (unsigned int)VEC);
                atomicAdd(acc.lo + dcell[0], lo);
                atomicAdd(acc.hi + dcell[0], hi);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (dcell[e] >= 0) dep_add(acc, dcell[e], dq2[e]);
            }
        }
        *reinterpret_cast<V *>(X + base) = pack(xa, V{});
        *reinterpret_cast<V *>(VX + base) = pack(vxa, V{});
    }
    if (cur >= 0) flush(true);
    cp_async_wait_all();  // the groups issued past the block's last tile are empty; none is left writing
}

// ---------------------------------------------------------------- field solve
// The Poisson problem of Algorithm 3 (tridiagonal, constant coefficients,
// phi_0 = V(t), phi_{N_G-1} = 0) is solved through its exact prefix-sum form:
// with d_p = phi_{p+1} - phi_p, D_k = Q_i,k - Q_e,k (fixed-point densities,
// integers) and F_p = sum_{k=1..p} D_k, the discrete equation gives
// d_p = d_0 - c F_p, so phi_p = V + p d_0 - c G_p with G_p = sum_{j<p} F_j and
// phi_{N_G-1} = 0 fixes d_0 = (c G_M - V) / M (M = N_G - 1, c = dx^2 e
// FACTOR_W / (eps0 2^32)).  F and G_M are exact integer sums.  The field
// follows as E_p = -(d_{p-1} + d_p) / (2 dx) inside and from the one-sided
// forms with the half-cell charge at the electrodes; E needs only F and d_0.
//
// Each of the g threads of the group (named barrier `bar`) owns a run of
// consecutive grid points.
template <int G>
struct FieldScratch {
    long long w64[33];
    __int128 w128[32];
    double wd[33];
    double d0;
};

// Load (Q_e, Q_i) of the owned points; swap in the accumulated deposition
// when `swap` (and add the current field to the time sums when `measure`).
// The arrays are distinct (one discharge's grid blocks); the restrict
// qualifiers let every load be issued before the stores instead of one
// round trip per array.
template <int PMAX>
__device__ __forceinline__ void load_q_arrays(long long *__restrict__ q_e, long long *__restrict__ q_i,
                                              long long *__restrict__ acc_e, long long *__restrict__ acc_i,
                                              const long long *__restrict__ f_cur, double *__restrict__ sum_qe,
                                              double *__restrict__ sum_qi, double *__restrict__ sum_f, int first,
                                              int last, bool swap, bool next_ion, bool measure, long long *Qe,
                                              long long *Qi)
{
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        const int p = first + j;
        Qe[j] = 0;
        Qi[j] = 0;
        if (p >= last) continue;
        if (swap && measure) {
            sum_qe[p] += (double)q_e[p];
            sum_qi[p] += (double)q_i[p];
            sum_f[p] += (double)f_cur[p];
        }
        if (swap) {
            Qe[j] = acc_e[p];
            acc_e[p] = 0;
            q_e[p] = Qe[j];
            if (next_ion) {
                Qi[j] = acc_i[p];
                acc_i[p] = 0;
                q_i[p] = Qi[j];
            } else {
                Qi[j] = q_i[p];
            }
        } else {
            Qe[j] = q_e[p];
            Qi[j] = q_i[p];
        }
    }
}

template <int PMAX>
__device__ __forceinline__ void load_q(const DischargeDev &D, int first, int last, bool swap, bool next_ion,
                                       bool measure, long long *Qe, long long *Qi)
{
    load_q_arrays<PMAX>(D.q_e, D.q_i, D.acc_e, D.acc_i, D.f_cur, D.sum_qe, D.sum_qi, D.sum_f, first, last, swap,
                        next_ion, measure, Qe, Qi);
}

// Field of within-cycle step tc.  full: also densities n_e, n_i and phi.
template <typename T, int G>
__device__ void solve_field(const DischargeDev &D, long long tc, bool swap, bool next_ion, bool measure, bool full,
                            int gtid, int bar, FieldScratch<G> &sm)
{
    constexpr int PMAX = (EDUPIC_MAX_GRID + G - 1) / G;
    const int ng = D.ng, M = ng - 1;
    const int per = (ng + G - 1) / G;
    const int first = gtid * per, last = min(first + per, ng);
    if (swap && measure && gtid == 0) {
        D.fs->sum_V += D.fs->V;
        D.fs->sum_d0 += D.fs->d0;
    }
    const double V = D.vdrive[tc];  // read before the stores below
    long long Qe[PMAX], Qi[PMAX], F[PMAX];
    load_q<PMAX>(D, first, last, swap, next_ion, measure, Qe, Qi);
    // F: inclusive scan of D_p over p = 0..M (D_p = 0 at the electrodes)
    long long run = 0;
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        const int p = first + j;
        if (p >= 1 && p <= M - 1 && p < last) run += Qi[j] - Qe[j];
    }
    long long tot64;
    const long long off = group_excl_scan(run, sm.w64, tot64, gtid, G, bar);
    __int128 gpart = 0;
    {
        long long a = off;
#pragma unroll
        for (int j = 0; j < PMAX; ++j) {
            const int p = first + j;
            if (p >= last) break;
            if (p >= 1 && p <= M - 1) a += Qi[j] - Qe[j];
            F[j] = a;
            D.f_cur[p] = a;
            if (p <= M - 1) gpart += (__int128)a;
        }
    }
    const __int128 gtot = group_sum128(gpart, sm.w128, gtid, G, bar);
    const double c = D.poisson_c;
    if (gtid == 0) {
        const double d0 = (c * (double)gtot - V) / (double)M;
        sm.d0 = d0;
        D.fs->V = V;
        D.fs->d0 = d0;
    }
    bar_sync(bar, G);
    const double d0 = sm.d0;
    T *et = reinterpret_cast<T *>(D.ef_t);
    long long fprev = off;  // F_{first-1}
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        const int p = first + j;
        if (p >= last) break;
        double ef;
        if (p == 0)
            ef = -d0 * D.inv_dx - D.edge_c * (double)(Qi[j] - Qe[j]);
        else if (p < M)
            ef = -(2.0 * d0 - c * (double)(fprev + F[j])) * D.inv_2dx;
        else
            ef = -(d0 - c * (double)fprev) * D.inv_dx + D.edge_c * (double)(Qi[j] - Qe[j]);
        D.ef[p] = ef;
        et[p] = (T)ef;
        fprev = F[j];
    }
    if (!full) return;
    // densities (Algorithm 2, x2 at the half-volume edge points) and phi
    double gp = 0.0;
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        const int p = first + j;
        if (p < last && p <= M - 1) gp += (double)F[j];
    }
    double totd;
    const double offd = group_excl_scan(gp, sm.wd, totd, gtid, G, bar);
    double g = offd;
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        const int p = first + j;
        if (p >= last) break;
        double ne = D.factor_w * ((double)Qe[j] * (1.0 / 4294967296.0));
        double ni = D.factor_w * ((double)Qi[j] * (1.0 / 4294967296.0));
        if (p == 0 || p == M) {
            ne *= 2.0;
            ni *= 2.0;
        }
        D.n_e[p] = ne;
        D.n_i[p] = ni;
        D.phi[p] = p == 0 ? V : (p == M ? 0.0 : V + (double)p * d0 - c * g);
        g += (double)F[j];
    }
}

// ---------------------------------------------------------------- compaction
// Bitonic sort of n ints in shared memory by a group of g threads.
__device__ __forceinline__ void group_sort(int *a, int n, int gtid, int g, int bar)
{
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = n + gtid; i < m; i += g) a[i] = INT_MAX;
    bar_sync(bar, g);
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = gtid; i < m; i += g) {
                const int l = i ^ j;
                if (l > i) {
                    const int ai = a[i], al = a[l];
                    const bool up = (i & k) == 0;
                    if ((ai > al) == up) {
                        a[i] = al;
                        a[l] = ai;
                    }
                }
            }
            bar_sync(bar, g);
        }
    }
}

// Sorted copy of an event list: in shared memory when it fits (sA), else in
// the discharge's global sort buffer (bitonic sort; its length is padded to
// a power of two <= kEvents).  Returns the sorted array.
__device__ __forceinline__ int *sorted_events(const DischargeDev &D, const int *src, int n, int *sA, int gtid, int g,
                                              int bar)
{
    int *a = n <= kSortShared ? sA : D.sort_buf;
    for (int i = gtid; i < n; i += g) a[i] = src[i];
    group_sort(a, n, gtid, g, bar);
    return a;
}

// Holes of species sp sorted ascending, then filled by the tail survivors
// [N', N) in ascending order (the canonical removal order).
template <typename T>
__device__ long long compact_species(const DischargeDev &D, int sp, int *sA, int *sW, int gtid, int g, int bar)
{
    Ctrl *C = D.ctrl;
    const long long n = C->n[sp];
    int H = C->holes[sp];
    if (H > kEvents) H = kEvents;  // error bit already set by k_push
    if (H == 0) return n;
    const int *hs = sorted_events(D, D.holes[sp], H, sA, gtid, g, bar);
    const long long nn = n - H;
    T *X = reinterpret_cast<T *>(D.x[sp]);
    T *VX = reinterpret_cast<T *>(D.vx[sp]);
    T *VY = reinterpret_cast<T *>(D.vy[sp]);
    T *VZ = reinterpret_cast<T *>(D.vz[sp]);
    const T L = is_f64<T>() ? (T)D.L : (T)D.Lf;
    int filled = 0;
    for (int b = 0; b < H; b += g) {
        const long long j = nn + b + gtid;
        bool alive = false;
        if (b + gtid < H) {
            const T xj = X[j];
            alive = (xj >= (T)0.0) && (xj <= L);
        }
        int tot;
        const int r = group_excl_scan(alive ? 1 : 0, sW, tot, gtid, g, bar);
        const int k = filled + r;
        const int dst = (alive && k < H) ? hs[k] : -1;
        if (alive && (dst < 0 || dst >= nn)) atomicOr(&C->error, kErrHoles);  // inconsistent hole list
        if (alive && dst >= 0 && dst < nn) {
            X[dst] = X[j];
            VX[dst] = VX[j];
            VY[dst] = VY[j];
            VZ[dst] = VZ[j];
        }
        filled += tot;
    }
    bar_sync(bar, g);
    return nn;
}

// Ionisation products appended in ascending parent order.
template <typename T>
__device__ void append_products(const DischargeDev &D, int *sA, long long &ne, long long &ni, int gtid, int g, int bar)
{
    Ctrl *C = D.ctrl;
    int P = C->products;
    if (P > kEvents) P = kEvents;
    if (P == 0) return;
    const int *ps = sorted_events(D, D.prod_parent, P, sA, gtid, g, bar);
    long long room = D.cap[0] - ne;
    if (D.cap[1] - ni < room) room = D.cap[1] - ni;
    const long long keep = (long long)P < room ? (long long)P : (room > 0 ? room : 0);
    T *X0 = reinterpret_cast<T *>(D.x[0]), *X1 = reinterpret_cast<T *>(D.x[1]);
    T *VX0 = reinterpret_cast<T *>(D.vx[0]), *VX1 = reinterpret_cast<T *>(D.vx[1]);
    T *VY0 = reinterpret_cast<T *>(D.vy[0]), *VY1 = reinterpret_cast<T *>(D.vy[1]);
    T *VZ0 = reinterpret_cast<T *>(D.vz[0]), *VZ1 = reinterpret_cast<T *>(D.vz[1]);
    const T *px = reinterpret_cast<const T *>(D.prod_x);
    for (int i = gtid; i < P; i += g) {
        const int h = D.prod_parent[i];
        int lo = 0, hi = P;  // rank of h among the sorted parents
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ps[mid] < h)
                lo = mid + 1;
            else
                hi = mid;
        }
        const int r = lo;
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
    if (gtid == 0) {
        C->counters[EDUPIC_C_CREATED] += (unsigned long long)keep;
        if (keep < (long long)P) {
            C->counters[EDUPIC_C_DROPPED] += (unsigned long long)(P - keep);
            C->error |= kErrCapacity;
        }
    }
    ne += keep;
    ni += keep;
    bar_sync(bar, g);
}

// Secondary electrons of the step (Sec. 5) appended after the ionisation
// pairs, in ascending order of the emitting ion's slot (each ion emits at
// most once per step, so the order is unique).
template <typename T>
__device__ void append_emitted(const DischargeDev &D, int *sA, long long &ne, int gtid, int g, int bar)
{
    Ctrl *C = D.ctrl;
    int M = C->emitted;
    if (M > kEvents) M = kEvents;  // error bit already set by k_push
    if (M == 0) return;
    const int *ps = sorted_events(D, D.emit_parent, M, sA, gtid, g, bar);
    const long long room = D.cap[0] - ne;
    const long long keep = (long long)M < room ? (long long)M : (room > 0 ? room : 0);
    T *X0 = reinterpret_cast<T *>(D.x[0]);
    T *VX0 = reinterpret_cast<T *>(D.vx[0]);
    T *VY0 = reinterpret_cast<T *>(D.vy[0]);
    T *VZ0 = reinterpret_cast<T *>(D.vz[0]);
    for (int i = gtid; i < M; i += g) {
        const int h = D.emit_parent[i];
        int lo = 0, hi = M;  // rank of h among the sorted emitters
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ps[mid] < h)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo < keep) {
            const long long se = ne + lo;
            X0[se] = reinterpret_cast<const T *>(D.emit_x)[i];
            VX0[se] = reinterpret_cast<const T *>(D.emit_v[0])[i];
            VY0[se] = reinterpret_cast<const T *>(D.emit_v[1])[i];
            VZ0[se] = reinterpret_cast<const T *>(D.emit_v[2])[i];
        }
    }
    if (gtid == 0) {
        if (keep < (long long)M) {
            C->counters[EDUPIC_C_DROPPED] += (unsigned long long)(M - keep);
            C->error |= kErrCapacity;
        }
    }
    ne += keep;
    bar_sync(bar, g);
}

template <typename T>
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const DischargeDev *__restrict__ DD, int nd,
                                                               int ion_step, int measure)
{
    __shared__ int sA[kSortShared];
    __shared__ int sW[33];
    __shared__ FieldScratch<kGroupB> sF;
    __shared__ long long sN[2];
    __shared__ DischargeDev D;
    {
        // the descriptor is staged in shared memory before the wait
        const int *src = reinterpret_cast<const int *>(DD + blockIdx.x);
        int *dst = reinterpret_cast<int *>(&D);
        for (int i = threadIdx.x; i < (int)(sizeof(DischargeDev) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    pdl_wait();
    pdl_launch_next();
    if (!D.active || D.ctrl->step >= D.stop_step) return;
    Ctrl *C = D.ctrl;
    const long long next = C->step + 1;
    if (threadIdx.x < kGroupA) {
        // (A) particle bookkeeping
        const int gtid = threadIdx.x;
        long long ne = compact_species<T>(D, 0, sA, sW, gtid, kGroupA, 1);
        long long ni = ion_step ? compact_species<T>(D, 1, sA, sW, gtid, kGroupA, 1) : C->n[1];
        append_products<T>(D, sA, ne, ni, gtid, kGroupA, 1);
        if (ion_step) append_emitted<T>(D, sA, ne, gtid, kGroupA, 1);
        if (gtid == 0) {
            sN[0] = ne;
            sN[1] = ni;
        }
    } else {
        // (B) density swap, diagnostics, field of the next step
        const int gb = threadIdx.x - kGroupA;
        if (measure && D.nxt > 0) {
            // xt sums of the grid quantities of this step, before the swap
            const int b = (int)((C->step % D.nt) / D.nbin);
            for (int p = gb; p < D.ng; p += kGroupB) {
                const size_t j = (size_t)p * D.nxt + b;
                D.xt_f[j] += (double)D.f_cur[p];
                D.xt_qe[j] += (double)D.q_e[p];
                D.xt_qi[j] += (double)D.q_i[p];
                if (ion_step) D.xt_cnti[j] += (double)D.q_i[p];
            }
            if (gb == 0) {
                D.xt_V[b] += D.fs->V;
                D.xt_d0[b] += D.fs->d0;
                D.xt_steps[b] += 1;
                if (ion_step) D.xt_steps[D.nxt + b] += 1;
            }
            bar_sync(2, kGroupB);
        }
        const long long tc = next % D.nt;
        solve_field<T, kGroupB>(D, tc, true, (tc % D.nsub) == 0, measure != 0, false, gb, 2, sF);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        C->n[0] = sN[0];
        C->n[1] = sN[1];
        C->holes[0] = 0;
        C->holes[1] = 0;
        C->products = 0;
        C->emitted = 0;
        C->step = next;
        if (measure) C->measured += 1;
    }
}

// ---------------------------------------------------------------- periodic cell sort
// Every sort_every ion subcycles, after the step that reaches a multiple of
// sort_every * N_SUB, each species is put in ascending order of its
// deposition cell, keeping the slot order within a cell (a stable counting
// sort), so that the particles a warp reads next share few cells.  The slot,
// and with it the random-number counter, follows the new order.  Four
// launches per species, each over the chunks of kSortChunk particles of
// every discharge that is due: chunk histograms, their scan into the first
// slot of every (cell, chunk), the stable scatter into a scratch copy, and
// the copy back.  Idempotent: a discharge that stays at a due step (a
// finished request) is sorted again without change.
__device__ __forceinline__ bool sort_due(const DischargeDev &D, int sp)
{
    if (!D.active || D.sort_every <= 0) return false;
    const long long s = D.ctrl->step;
    return s > 0 && s % ((long long)D.sort_every * D.nsub) == 0 && D.ctrl->n[sp] > 1;
}

// Chunks of the due discharges -> exclusive prefix sPre[0..nd] in shared memory.
__device__ __forceinline__ void sort_chunk_prefix(const DischargeDev *DD, int nd, int sp, int *sPre, int *sW)
{
    int running = 0;
    for (int base = 0; base < nd; base += blockDim.x) {
        const int d = base + threadIdx.x;
        int cnt = 0;
        if (d < nd && sort_due(DD[d], sp)) cnt = (int)((DD[d].ctrl->n[sp] + kSortChunk - 1) / kSortChunk);
        int tot;
        const int ex = group_excl_scan(cnt, sW, tot, threadIdx.x, blockDim.x, 1);
        if (d < nd) sPre[d] = running + ex;
        running += tot;
    }
    if (threadIdx.x == 0) sPre[nd] = running;
    __syncthreads();
}

__device__ __forceinline__ int sort_owner(const int *sPre, int nd, int chunk)  // discharge of a global chunk
{
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sPre[mid] <= chunk)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Pass 1: per chunk, the count of particles in each cell ([chunk][ng]).
template <typename T>
__global__ void __launch_bounds__(256) k_sort_count(const DischargeDev *__restrict__ DD, int nd, int sp, int ng_max)
{
    extern __shared__ __align__(16) unsigned int sHist[];  // [warps][ng_max], then the chunk prefix
    int *sPre = reinterpret_cast<int *>(sHist + (blockDim.x / 32) * ng_max);
    __shared__ int sW[33];
    sort_chunk_prefix(DD, nd, sp, sPre, sW);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int *h = sHist + warp * ng_max;
    const int total = sPre[nd];
    for (int chunk = blockIdx.x * (blockDim.x / 32) + warp; chunk < total; chunk += gridDim.x * (blockDim.x / 32)) {
        const int d = sort_owner(sPre, nd, chunk);
        const DischargeDev &D = DD[d];
        const int ng = D.ng;
        const long long n = D.ctrl->n[sp];
        const long long base = (long long)(chunk - sPre[d]) * kSortChunk;
        const T *X = reinterpret_cast<const T *>(D.x[sp]);
        const T inv_dx = is_f64<T>() ? (T)D.inv_dx : (T)D.inv_dxf;
        for (int p = lane; p < ng; p += 32) h[p] = 0u;
        __syncwarp();
        for (int k = lane; k < kSortChunk; k += 32) {
            const long long j = base + k;
            if (j >= n) break;
            T c0;
            atomicAdd(h + cell<T>(X[j], inv_dx, ng, c0), 1u);
        }
        __syncwarp();
        unsigned int *out = D.sort_cnt + (size_t)(chunk - sPre[d]) * ng;
        for (int p = lane; p < ng; p += 32) out[p] = h[p];
        __syncwarp();
    }
}

// Pass 2 (one block per discharge): counts -> first slot of every (cell,
// chunk): cells in ascending order, chunks (slot order) within a cell.
template <typename T>
__global__ void __launch_bounds__(256) k_sort_scan(const DischargeDev *__restrict__ DD, int sp)
{
    extern __shared__ __align__(16) unsigned int sTot[];  // [ng_max]
    __shared__ unsigned int sW[33];
    const DischargeDev &D = DD[blockIdx.x];
    if (!sort_due(D, sp)) return;
    const int ng = D.ng;
    const int nch = (int)((D.ctrl->n[sp] + kSortChunk - 1) / kSortChunk);
    unsigned int *cnt = D.sort_cnt;
    for (int p = threadIdx.x; p < ng; p += blockDim.x) {
        unsigned int t = 0;
        for (int c = 0; c < nch; ++c) t += cnt[(size_t)c * ng + p];
        sTot[p] = t;
    }
    __syncthreads();
    // exclusive prefix over the cells (each thread a run of consecutive cells)
    const int per = (ng + blockDim.x - 1) / blockDim.x;
    const int first = threadIdx.x * per, last = min(first + per, ng);
    unsigned int run = 0;
    for (int p = first; p < last; ++p) run += sTot[p];
    unsigned int tot;
    unsigned int off = group_excl_scan(run, sW, tot, threadIdx.x, blockDim.x, 1);
    for (int p = first; p < last; ++p) {
        const unsigned int v = sTot[p];
        sTot[p] = off;
        off += v;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < ng; p += blockDim.x) {
        unsigned int r = sTot[p];
        for (int c = 0; c < nch; ++c) {
            const unsigned int v = cnt[(size_t)c * ng + p];
            cnt[(size_t)c * ng + p] = r;
            r += v;
        }
    }
}

// Pass 3: every chunk's particles, in slot order, to the next free slot of
// their cell in the scratch copy (a warp takes 32 slots at a time; lanes in
// the same cell are ranked by lane).
template <typename T>
__global__ void __launch_bounds__(256) k_sort_scatter(const DischargeDev *__restrict__ DD, int nd, int sp, int ng_max)
{
    extern __shared__ __align__(16) unsigned int sRun[];  // [warps][ng_max], then the chunk prefix
    int *sPre = reinterpret_cast<int *>(sRun + (blockDim.x / 32) * ng_max);
    __shared__ int sW[33];
    sort_chunk_prefix(DD, nd, sp, sPre, sW);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int *run = sRun + warp * ng_max;
    const int total = sPre[nd];
    for (int chunk = blockIdx.x * (blockDim.x / 32) + warp; chunk < total; chunk += gridDim.x * (blockDim.x / 32)) {
        const int d = sort_owner(sPre, nd, chunk);
        const DischargeDev &D = DD[d];
        const int ng = D.ng;
        const long long n = D.ctrl->n[sp];
        const long long base = (long long)(chunk - sPre[d]) * kSortChunk;
        const T *src[4] = {reinterpret_cast<const T *>(D.x[sp]), reinterpret_cast<const T *>(D.vx[sp]),
                           reinterpret_cast<const T *>(D.vy[sp]), reinterpret_cast<const T *>(D.vz[sp])};
        T *dst[4] = {reinterpret_cast<T *>(D.sort_tmp[0]), reinterpret_cast<T *>(D.sort_tmp[1]),
                     reinterpret_cast<T *>(D.sort_tmp[2]), reinterpret_cast<T *>(D.sort_tmp[3])};
        const T inv_dx = is_f64<T>() ? (T)D.inv_dx : (T)D.inv_dxf;
        const unsigned int *first = D.sort_cnt + (size_t)(chunk - sPre[d]) * ng;
        for (int p = lane; p < ng; p += 32) run[p] = first[p];
        __syncwarp();
        for (int k = 0; k < kSortChunk; k += 32) {
            const long long j = base + k + lane;
            const bool act = j < n;
            const unsigned int mask = __ballot_sync(0xffffffffu, act);
            if (mask == 0u) break;
            int p = 0;
            unsigned int peers = 0u, rank = 0u;
            if (act) {
                T c0;
                const T x = src[0][j];
                p = cell<T>(x, inv_dx, ng, c0);
                peers = __match_any_sync(mask, p);
                rank = (unsigned int)__popc(peers & ((1u << lane) - 1u));
                const unsigned int o = run[p] + rank;
                if (o < (unsigned long long)n) {
                    dst[0][o] = x;
                    dst[1][o] = src[1][j];
                    dst[2][o] = src[2][j];
                    dst[3][o] = src[3][j];
                } else {
                    atomicOr(&D.ctrl->error, kErrHoles);  // inconsistent counts (never expected)
                }
            }
            __syncwarp();
            if (act && rank == 0u) run[p] += (unsigned int)__popc(peers);
            __syncwarp();
        }
    }
}

// Pass 4: the sorted scratch copy back into the particle arrays.
template <typename T>
__global__ void __launch_bounds__(256) k_sort_copy(const DischargeDev *__restrict__ DD, int nd, int sp)
{
    extern __shared__ __align__(16) int sPreC[];  // chunk prefix
    __shared__ int sW[33];
    sort_chunk_prefix(DD, nd, sp, sPreC, sW);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = sPreC[nd];
    for (int chunk = blockIdx.x * (blockDim.x / 32) + warp; chunk < total; chunk += gridDim.x * (blockDim.x / 32)) {
        const int d = sort_owner(sPreC, nd, chunk);
        const DischargeDev &D = DD[d];
        const long long n = D.ctrl->n[sp];
        const long long base = (long long)(chunk - sPreC[d]) * kSortChunk;
        void *arr[4] = {D.x[sp], D.vx[sp], D.vy[sp], D.vz[sp]};
        for (int a = 0; a < 4; ++a) {
            const T *s = reinterpret_cast<const T *>(D.sort_tmp[a]);
            T *o = reinterpret_cast<T *>(arr[a]);
            for (int k = lane; k < kSortChunk; k += 32) {
                const long long j = base + k;
                if (j >= n) break;
                o[j] = s[j];
            }
        }
    }
}

// init(N_INIT) of Algorithm 1: n particles of species sp of discharge d at
// rest at x = L R01, R01 from block 9 of each slot's counter (current step);
// sets the count.
template <typename T>
__global__ void k_seed(const DischargeDev *__restrict__ DD, int d, int sp, long long n)
{
    const DischargeDev &D = DD[d];
    const unsigned long long s = (unsigned long long)D.ctrl->step;
    const RngKey key{(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)D.seed, (uint32_t)(D.seed >> 32)};
    T *X = reinterpret_cast<T *>(D.x[sp]);
    T *VX = reinterpret_cast<T *>(D.vx[sp]);
    T *VY = reinterpret_cast<T *>(D.vy[sp]);
    T *VZ = reinterpret_cast<T *>(D.vz[sp]);
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        double u, u_unused;
        draw<double>(key, (uint32_t)j, sp, 9, u, u_unused);
        X[j] = (T)(D.L * u);
        VX[j] = (T)0;
        VY[j] = (T)0;
        VZ[j] = (T)0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) D.ctrl->n[sp] = n;
}

// Densities of one species from its particles (after a load), into q and,
// for ions between ion steps, also into the pending accumulator.
template <typename T>
__global__ void k_deposit(const DischargeDev *__restrict__ DD, int d, int sp, int also_acc)
{
    const DischargeDev &D = DD[d];
    const long long n = D.ctrl->n[sp];
    const T *X = reinterpret_cast<const T *>(D.x[sp]);
    const T inv_dx = is_f64<T>() ? (T)D.inv_dx : (T)D.inv_dxf;
    long long *q = sp == 0 ? D.q_e : D.q_i;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        T c0;
        const int p = cell<T>(X[j], inv_dx, D.ng, c0);
        const unsigned long long q2 = split_q2(c0 - (T)p);
        atomicAdd(reinterpret_cast<unsigned long long *>(q + p), 4294967296ull - q2);
        atomicAdd(reinterpret_cast<unsigned long long *>(q + p + 1), q2);
        if (also_acc) {
            atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_i + p), 4294967296ull - q2);
            atomicAdd(reinterpret_cast<unsigned long long *>(D.acc_i + p + 1), q2);
        }
    }
}

// Densities, potential and field of the current step from q_e / q_i.
template <typename T>
__global__ void __launch_bounds__(kGroupB) k_fields(const DischargeDev *__restrict__ DD, int d)
{
    __shared__ FieldScratch<kGroupB> sF;
    const DischargeDev &D = DD[d];
    const long long tc = D.ctrl->step % D.nt;
    solve_field<T, kGroupB>(D, tc, false, false, false, true, threadIdx.x, 2, sF);
}

// Time averages over the measured steps into D.avg: n_e, n_i from the summed
// fixed-point densities, phi from the summed V, d_0 and F through the same
// prefix-sum form (sum_t phi_p = S_V + p S_d0 - c sum_{j<p} S_F,j).
template <typename T>
__global__ void __launch_bounds__(kGroupB) k_averages(const DischargeDev *__restrict__ DD, int d)
{
    __shared__ double sWd[33];
    constexpr int PMAX = (EDUPIC_MAX_GRID + kGroupB - 1) / kGroupB;
    const DischargeDev &D = DD[d];
    const int ng = D.ng, M = ng - 1, gtid = threadIdx.x;
    const int per = (ng + kGroupB - 1) / kGroupB;
    const int first = gtid * per, last = min(first + per, ng);
    const long long m = D.ctrl->measured;
    const double inv_m = m > 0 ? 1.0 / (double)m : 0.0;
    double run = 0.0;
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        const int p = first + j;
        if (p < last && p <= M - 1) run += D.sum_f[p];
    }
    double tot;
    double g = group_excl_scan(run, sWd, tot, gtid, kGroupB, 2);
    const double c = D.poisson_c, SV = D.fs->sum_V, Sd0 = D.fs->sum_d0;
    double *ne = D.avg, *ni = D.avg + ng, *phi = D.avg + 2 * ng;
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        const int p = first + j;
        if (p >= last) break;
        const double edge = (p == 0 || p == M) ? 2.0 : 1.0;
        ne[p] = edge * D.factor_w * (D.sum_qe[p] * (1.0 / 4294967296.0)) * inv_m;
        ni[p] = edge * D.factor_w * (D.sum_qi[p] * (1.0 / 4294967296.0)) * inv_m;
        phi[p] = p == M ? 0.0 : (SV + (double)p * Sd0 - c * g) * inv_m;
        if (p <= M - 1) g += D.sum_f[p];
    }
}

}  // namespace edupic
