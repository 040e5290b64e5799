// Internal structures shared by the host orchestration and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/edupic.h"

namespace edupic {

constexpr int kFinalizeThreads = 512;  // one CTA per discharge for compaction + field solve
constexpr int kGroupA = 128;           // finalize threads doing compaction and append
constexpr int kGroupB = kFinalizeThreads - kGroupA;  // finalize threads doing the field solve
constexpr int kEvents = EDUPIC_STEP_EVENTS;
constexpr int kPushShapeCount = EDUPIC_PUSH_SHAPES;  // launch shapes of the particle kernel the autotuner chooses among
constexpr int kSortShared = 8192;      // event lists up to this size are sorted in shared memory
constexpr int kCoarse = 2048;          // entries of the coarse sigma_max tables (shared memory)
constexpr int kSortChunk = 2048;       // particles per chunk (one warp) of the periodic cell sort
constexpr int kEepfStripes = 16;       // copies of the EEPF histogram the particle kernel spreads its atomics over
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // limit of every bounded device wait (1 s)

// Launch shapes of the particle kernel: threads per block, tiles in the
// shared-memory ring, and the blocks per SM the register budget is set for
// (__launch_bounds__).  The autotuner times the shapes on the live workload;
// every shape gives the same results (the arithmetic of a slot does not
// depend on which block or warp takes it, and deposition is exact).  A tile
// is threads x VEC particles (VEC = one Philox block's test uniforms per
// thread: 4 in FP32, 2 in FP64); tiles stay within the 1024-particle
// padding of the particle arrays.
struct PushShape {
    int threads, stages, min_blocks;
};
__host__ __device__ constexpr PushShape push_shape_of(bool f64, int s)
{
    return f64 ? (s == 0 ? PushShape{256, 3, 2} : s == 1 ? PushShape{256, 2, 2}
                  : s == 2 ? PushShape{128, 3, 3} : PushShape{128, 2, 4})
               : (s == 0 ? PushShape{256, 4, 2} : s == 1 ? PushShape{256, 3, 2}
                  : s == 2 ? PushShape{128, 3, 4} : PushShape{256, 2, 3});
}

// Device error bits (ctrl->error).
enum : int {
    kErrHoles = 1,     // more absorbed particles in a step than kEvents
    kErrProducts = 2,  // more ionisations in a step than kEvents
    kErrCapacity = 4,  // created pairs dropped at particle capacity
    kErrNan = 8,       // non-finite position
    kErrTimeout = 16,  // a bounded device wait expired (the wait self-test)
};

// Per-discharge counters and counts, written by the kernels.
struct Ctrl {
    long long n[2];         // live particles per species
    long long step;         // global step index s
    long long measured;     // steps accumulated into the diagnostics
    int holes[2];           // absorbed particles of the current step, per species
    int products;           // ionisations of the current step
    int error;              // kErr* bits
    int emitted;            // secondary electrons of the current step
    int pad;
    unsigned long long counters[EDUPIC_N_COUNTERS];
};

// Scalars of the current field and their time sums (diagnostics).
struct FieldState {
    double V, d0;       // drive voltage and d_0 = phi_1 - phi_0 of the current field
    double sum_V, sum_d0;
};

// Cross-section tables in particle precision T: sigsum[k] = sum of the
// process cross sections (n*sigma_tot is formed in the kernel as
// sigsum * n_gas), thr[k] = cumulative process fractions (thr1, thr2).
// Everything a kernel needs about one discharge (in device memory).
struct DischargeDev {
    // constants (FP64 values; FP32 copies below)
    double L, dx, inv_dx, dt_e, dt_i, factor_w, factor_e, factor_i, n_gas, sig_th;
    double half_me, half_mar, half_mu_e, half_mu_arar, mu_e, ar_mass, e_exc, e_ion;
    double eepf_lo, eepf_hi, eepf_de, ifed_de, cs_de_e, cs_de_i;
    double poisson_c;   // dx^2 e FACTOR_W / (eps0 2^32): f_p = c (Q_i - Q_e)
    double rho_c;       // e FACTOR_W / 2^32
    double harm_freq[EDUPIC_MAX_HARMONICS];
    double harm_volt[EDUPIC_MAX_HARMONICS];
    double refl_eta[2], see_gamma[2];  // surface processes per electrode (0 = off)
    double see_sth;                    // thermal speed sqrt(T_see e / m_e) of emitted electrons
    double nu_star[2], p_star[2];      // null-collision bound nu* and P* = 1 - exp(-nu* dt), per species
    float Lf, inv_dxf, dt_ef, dt_if, factor_ef, factor_if, n_gasf, sig_thf;
    float e_of_v2_ef, e_of_v2_if, e_of_g2_if, mu_ef, e_excf, e_ionf;
    float eepf_lof, eepf_hif, inv_eepf_def, inv_ifed_def, inv_cs_de_ef, inv_cs_de_if;
    float ndt_ef, ndt_if;  // n_gas * dt (electrons, ions)
    float e_idx_ef;        // (m_e / 2e) / DE_CS: table index of v^2
    float g_idx_if;        // (mu / 2e) / DE_CS: table index of g^2
    float refl_etaf[2], see_gammaf[2], see_sthf;
    float p_starf[2];   // P* in FP32
    float null_ratf[2]; // n_gas / nu*: nu / nu* = sigsum v null_ratf
    // bound of the Ar+ direct collision test: the partner's largest speed
    // (gcap) and the squared speed at the top of the table's last entry
    double v2top[2], gcap;
    float v2topf[2], gcapf;
    double inv_2dx;
    double edge_c;     // e FACTOR_W * 2 / 2^32 * dx / (2 eps0): edge term of E from Q_i - Q_e
    int ng, nt, nsub, n_harm, eepf_bins, ifed_bins, cs_n_e, cs_n_i;
    int active;
    int null_coll;  // null-collision method: bit 0 electrons, bit 1 ions
    int nxt, nbin;  // xt diagnostics: time bins per cycle and steps per bin (nxt = 0: off)
    int sort_every;  // periodic cell sort: every sort_every ion subcycles (0: off)
    int pad_sort;
    long long stop_step;       // the discharge is frozen (skipped) once its step count reaches this
    long long cap[2];
    unsigned long long seed;
    // particle SoA (T = float or double)
    void *x[2], *vx[2], *vy[2], *vz[2];
    long long pstride[2];  // bytes from x to vx, vx to vy and vy to vz (the arena spaces them equally)
    // grid (FP64 unless noted)
    long long *q_e, *q_i;      // deposition sums used by the current step
    long long *acc_e, *acc_i;  // deposition of the next step (ions: next ion step)
    double *n_e, *n_i, *phi, *ef;
    void *ef_t;                // field in particle precision
    long long *f_cur;          // F_p of the current field (exact prefix sums of Q_i - Q_e)
    FieldState *fs;            // V and d_0 of the current field, and their time sums
    double *sum_qe, *sum_qi, *sum_f;  // time sums of Q_e, Q_i, F over the measured steps
    double *avg;               // [3][ng] read-back buffer: time-averaged n_e, n_i, phi
    unsigned long long *eepf;  // [kEepfStripes][eepf_bins], summed on read
    unsigned long long *ifed_pow, *ifed_gnd;
    double *power;             // [2] e-, Ar+: sum over measured pushes of E_x (v_old + v_new)
    // xt diagnostics, [ng][nxt] sums over the measured steps of each time bin:
    // F, Q_e, Q_i (all steps), Q_i of the ion steps, sum w v_c,x and sum w
    // eps_c (eV) per species, ionisation weights; [nxt] sums of V and d_0;
    // [2][nxt] measured steps (all, ion steps).  Null when off.
    double *xt_f, *xt_qe, *xt_qi, *xt_cnti, *xt_v[2], *xt_en[2], *xt_ion, *xt_V, *xt_d0;
    long long *xt_steps;
    Ctrl *ctrl;
    int *holes[2];
    int *prod_parent;
    int *emit_parent;          // emitting ion slot of each secondary electron (null without emission)
    void *emit_x, *emit_v[3];  // secondary electrons of the step (T)
    int *sort_buf;             // kEvents ints: global sort buffer for event lists above kSortShared
    void *prod_x, *prod_ve[3], *prod_vi[3];
    const void *cs_sig[2];     // T[cs_n]
    const void *cs_thr[2];     // T2[cs_n]
    // T[kCoarse]: Ar+: max of cs_sig over 2^cs_shift consecutive entries, rounded up;
    // e-: max of cs_sig_k times the bucket's top speed over the entries a v^2 of
    // each bucket (lv_bucket) can index, rounded up (the last bucket: +inf)
    const void *cs_max[2];
    const void *cs_pm[2];      // T[kCoarse]: max of cs_sig_k v_k over every entry up to the end of each block
    int cs_shift[2];
    int lv_base, lv_n;         // e-: first v^2 bucket of cs_max[0] and the number of buckets
    const double *vdrive;      // V(t) at the N_T steps of one cycle
    // periodic cell sort (sort_every > 0): [chunk][ng] counts, then first
    // slots, of kSortChunk-particle chunks; scratch copy of one species (T)
    unsigned int *sort_cnt;
    void *sort_tmp[4];
};

// Launchers implemented per precision (kernels_f32.cu / kernels_f64.cu).
template <typename T>
struct Launch {
    static cudaError_t deposit(const DischargeDev *dd, int nd, int d, int species, int also_acc, cudaStream_t st);
    static cudaError_t seed(const DischargeDev *dd, int d, int species, long long n, cudaStream_t st);
    static cudaError_t fields(const DischargeDev *dd, int nd, int d, cudaStream_t st);
    static cudaError_t averages(const DischargeDev *dd, int nd, int d, cudaStream_t st);
    // xt: the instantiation that accumulates the xt diagnostics (measured steps);
    // shape: launch shape of the others (0..kPushShapes-1, see push_shape)
    // sorted: some launched discharge keeps cell order (the warp-level deposition variant)
    static cudaError_t push(const DischargeDev *dd, int nd, int species, int measure, int grid, int ng_max,
                            int eepf_max, int null_any, int xt, int shape, int sorted, cudaStream_t st);
    static cudaError_t finalize(const DischargeDev *dd, int nd, int ion_step, int measure, cudaStream_t st);
    // one block waiting on a barrier that is never armed, for limit_ns (sets kErrTimeout in *err)
    static cudaError_t wait_expiry(unsigned long long limit_ns, int *err, cudaStream_t st);
    // periodic cell sort of both species of every discharge due at its current step
    static cudaError_t sort(const DischargeDev *dd, int nd, int ng_max, int sms, cudaStream_t st);
    static size_t push_smem(int nd, int ng_max, int eepf_max, int xt, int shape);
    static int push_blocks_per_sm(int species, size_t smem, int xt, int shape);
    static int push_threads(int xt, int shape);
};

}  // namespace edupic
