/*
 * edupic_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the 1D3V
 * electrostatic PIC/MCC particle loop for argon CCPs (Donko et al., "eduPIC:
 * an introductory particle based code for radio-frequency plasma simulation",
 * arXiv 2103.09642).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only the tests, the package's smoke check and bench.py's
 * CPU baseline leg and reference arm use it.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * Besides the particle loop of Sec. 2.1 it covers: init(N_INIT) of
 * Algorithm 1, the diagnostics of Sec. 3.5 (time averages, EEPF, IFED, power
 * absorption, the spatio-temporal "xt" maps), the null-collision method of
 * Sec. 2.1.6, and the extensions Sec. 5 proposes (ion-induced secondary
 * electrons, elastic electron reflection, a DC self-bias).
 *
 * Each function follows the paper's equations and algorithms in the paper's
 * order, one particle at a time, with no blocking, fusion or reordering beyond
 * what is noted.  Each point the paper leaves open is marked "Reading:" with
 * the choice made and its reason.
 *
 * Parity pins: every function here is pinned by a CPU test against a closed
 * form, an invariant, a textbook result, brute force or a published
 * known-answer vector (tests/test_oracle_*.py).  The full discharge physics
 * (densities, EEPF, IFEDF of the paper's figures) is "parity unpinned": the
 * Phelps cross-section fits the paper uses are not available, so a stand-in
 * cross-section set is passed in as input.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (no FMA contraction,
 * so x86-64 and aarch64 builds give identical results).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Physical constants (CODATA 2018, SI).  The paper uses SI units throughout  */
/* (Section 3.1) but does not list the values.                               */
/* ------------------------------------------------------------------------ */
#define ORC_E_CHARGE 1.602176634e-19
#define ORC_E_MASS 9.1093837015e-31
#define ORC_EPSILON0 8.8541878128e-12
#define ORC_K_BOLTZMANN 1.380649e-23
#define ORC_AMU 1.66053906660e-27
#define ORC_AR_MASS_U 39.948
#define ORC_EV_TO_J ORC_E_CHARGE
#define ORC_PI 3.14159265358979323846
#define ORC_OPAL_W_EV 10.0 /* Opal energy-sharing parameter for Ar, Sec. 2.1.6 */

#define ORC_MAX_HARM 4
#define ORC_SPECIES_E 0
#define ORC_SPECIES_I 1

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  The paper uses MT19937 (Section 3.3); this      */
/* build replaces it with a counter-based generator so that a particle's      */
/* random numbers depend only on (seed, slot, step, species, draw block).     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Uniform on [0,1) with 53 random bits from two 32-bit words. */
double orc_u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* Uniform on [0,1) with 24 random bits from one word (FP32 particle mode). */
float orc_u24(uint32_t a) { return (float)(a >> 8) * (1.0f / 16777216.0f); }

/* Random-number layout (the paper draws R01 from one sequential MT19937
 * stream, Sec. 3.3; any assignment of independent uniforms is equivalent).
 * Block 0 of counter word c0 = slot / 2 holds the collision-test uniforms of
 * the two slots 2k (words 0,1) and 2k+1 (words 2,3) (53 bits each; the FP32
 * particle mode takes 24-bit uniforms, four slots per block: see
 * orc_test_uniform_f32).  Blocks b >= 1 of
 * counter word c0 = slot hold the per-particle draws:
 *   e-:  1 (process, chi)  2 (eta, Opal)  3, 4 Box-Muller pairs of the new Ar+
 *   Ar+: 1, 2 Box-Muller pairs of the thermal partner  3 (process, chi)  4 (eta, -) */
static void philox_words(uint64_t seed, uint32_t c0, int64_t step, int species, int block, uint32_t w[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = c0;
    ctr[1] = (uint32_t)(uint64_t)step;
    ctr[2] = (uint32_t)((uint64_t)step >> 32);
    ctr[3] = ((uint32_t)species << 8) | (uint32_t)block;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, w);
}

/* Collision-test uniform of one slot (block 0, shared by slot pairs). */
static double test_uniform(uint64_t seed, int64_t slot, int64_t step, int species)
{
    uint32_t w[4];
    philox_words(seed, (uint32_t)((uint64_t)slot >> 1), step, species, 0, w);
    return (slot & 1) ? orc_u53(w[2], w[3]) : orc_u53(w[0], w[1]);
}

/* FP32 particle mode: block 0 of counter word slot / 4 serves four slots,
 * 24 bits from word slot % 4. */
float orc_test_uniform_f32(uint64_t seed, int64_t slot, int64_t step, int species)
{
    uint32_t w[4];
    philox_words(seed, (uint32_t)((uint64_t)slot >> 2), step, species, 0, w);
    return orc_u24(w[slot & 3]);
}

/* FP32 particle mode: 24-bit uniform from word `word` (0: a, 1: c) of the
 * per-particle block b >= 1, as the FP32 path draws (process, chi), (eta, opal). */
float orc_draw_u24(uint64_t seed, int64_t slot, int64_t step, int species, int block, int word)
{
    uint32_t w[4];
    philox_words(seed, (uint32_t)slot, step, species, block, w);
    return orc_u24(word == 0 ? w[0] : w[2]);
}

/* One per-particle Philox block (b >= 1) for (slot, global step, species). */
static void draw_block(uint64_t seed, int64_t slot, int64_t step, int species, int block, double u[2])
{
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = (uint32_t)slot;
    ctr[1] = (uint32_t)(uint64_t)step;
    ctr[2] = (uint32_t)((uint64_t)step >> 32);
    ctr[3] = ((uint32_t)species << 8) | (uint32_t)block;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, w);
    u[0] = orc_u53(w[0], w[1]);
    u[1] = orc_u53(w[2], w[3]);
}

/* Box-Muller: two standard normals from two uniforms on [0,1). */
static void box_muller(const double u[2], double z[2])
{
    double r = sqrt(-2.0 * log(1.0 - u[0]));
    double a = 2.0 * ORC_PI * u[1];
    z[0] = r * cos(a);
    z[1] = r * sin(a);
}

/* ------------------------------------------------------------------------ */
/* Parameters of one discharge (Table 1 and Table 2 quantities).             */
/* ------------------------------------------------------------------------ */
typedef struct {
    double gap_m;            /* L */
    double pressure_pa;      /* PRESSURE */
    double gas_temp_k;       /* TEMPERATURE */
    double area_m2;          /* electrode area A (1 cm^2 in the paper) */
    double weight;           /* W */
    int n_grid;              /* N_G */
    int steps_per_cycle;     /* N_T */
    int ion_subcycle;        /* N_SUB */
    double cycle_freq_hz;    /* frequency whose period is one RF cycle */
    int n_harm;              /* number of drive terms */
    double harm_freq_hz[ORC_MAX_HARM];
    double harm_volt_v[ORC_MAX_HARM];
    uint64_t seed;
    int eepf_bins;           /* N_EEPF */
    double eepf_de_ev;       /* DE_EEPF */
    int ifed_bins;           /* N_IFED */
    double ifed_de_ev;       /* DE_IFED */
    int64_t capacity;        /* MAX_N_P analogue, per species */
    double e_exc_ev;         /* lumped excitation threshold */
    double e_ion_ev;         /* ionisation threshold */
    /* surface processes (Sec. 5): ion-induced secondary electron yield and
     * elastic electron reflection probability, [0] powered, [1] grounded
     * electrode; temperature of the emitted electrons (eV) */
    double see_gamma[2];
    double refl_eta[2];
    double see_te_ev;
    /* null-collision method (Sec. 2.1.6, Sec. 5) instead of the per-particle
     * collision probability, per species: bit 0 electrons, bit 1 ions */
    int null_collision;
    /* spatio-temporal diagnostics (Sec. 3.5): time bins per RF cycle, 0 = off */
    int xt_bins;
    /* periodic cell sort of the particle arrays (not in the paper): every
     * sort_every ion subcycles, 0 = off */
    int sort_every;
} orc_params;

typedef struct {
    int64_t n;
    double *x, *vx, *vy, *vz;
} orc_species;

/* One created pair (ionisation): new electron and new ion at the parent's x. */
typedef struct {
    int64_t parent;
    double x, vxe, vye, vze, vxi, vyi, vzi;
} orc_product;

typedef struct {
    orc_params p;
    /* derived quantities (Section 3.1 / Algorithms 2-6) */
    double dx, inv_dx, dt_e, dt_i, factor_w, factor_e, factor_i, n_gas, ar_mass, mu_e, mu_arar, sigma_th_ar;
    /* cross sections (Section 3.2): per species, per process, per energy bin */
    int cs_n[2], cs_nproc[2];
    double cs_de[2];
    double *sigma[2];     /* [nproc][n] in m^2 */
    double *sigma_tot[2]; /* n * sigma_tot, [n] in 1/m (Section 3.2) */
    double nu_star[2];    /* null-collision frequency bound nu* per species (1/s) */
    double p_star[2];     /* P* = 1 - exp(-nu* dt) */
    orc_species sp[2];
    int64_t step;          /* global step counter s = c * N_T + t */
    int64_t *q_e, *q_i;    /* fixed-point deposition, 2^32 units per particle */
    double *n_e, *n_i, *rho, *phi, *efield;
    /* diagnostics */
    int64_t measured_steps;
    double *sum_ne, *sum_ni, *sum_phi;
    int64_t *eepf, *ifed_pow, *ifed_gnd;
    double work[2]; /* sum over measured pushes of q E_x v_c dt, per unit weight (J), e- and Ar+ */
    double v_bias;  /* DC voltage added at the powered electrode (Sec. 5 self-bias) */
    /* xt diagnostics (Sec. 3.5), [n_grid][xt_bins] sums over the measured steps
     * of each time bin: phi, E, n_e, n_i; per species the weighted sums of
     * v_c,x, of the energy (1/2) m |v_c|^2 in eV and of the weights; the
     * weighted ionisation events; and the number of measured steps per bin
     * (electrons and grid every step, ions on ion steps) */
    int nxt, nbin;
    double *xt_phi, *xt_ef, *xt_ne, *xt_ni, *xt_wv[2], *xt_we[2], *xt_w[2], *xt_ion;
    int64_t *xt_steps[2];
    int64_t counters[19];
    /* scratch */
    orc_product *prod;
    int64_t prod_cap;
    orc_product *emit; /* secondary electrons of this step (x, vxe, vye, vze; parent = ion slot) */
    unsigned char *absorbed;
    int error;
} orc_sim;

/* counter indices */
enum {
    ORC_C_ABS_E_POW = 0,
    ORC_C_ABS_E_GND,
    ORC_C_ABS_I_POW,
    ORC_C_ABS_I_GND,
    ORC_C_COLL_E_ELA,
    ORC_C_COLL_E_EXC,
    ORC_C_COLL_E_ION,
    ORC_C_COLL_I_ISO,
    ORC_C_COLL_I_BACK,
    ORC_C_SUBTHRESHOLD,
    ORC_C_CREATED,
    ORC_C_DROPPED,
    ORC_C_PUSH_E,
    ORC_C_PUSH_I,
    ORC_C_REFLECTED,
    ORC_C_EMITTED_POW,
    ORC_C_EMITTED_GND,
    ORC_C_NULL_TESTED,
    ORC_C_NULL_OVER
};

/* ------------------------------------------------------------------------ */
/* Step 1 -- charge assignment (Sec. 2.1.1, eqs. charge_assignment_1/2;      */
/* Algorithm 2).                                                             */
/* ------------------------------------------------------------------------ */

/* Grid index and the weight of grid point p+1 for a particle at x.
 * Reading: a particle exactly at x = L (c0 = N_G-1) is assigned to the last
 * cell with all weight on the last grid point. */
static void cell_of(double x, double inv_dx, int n_g, int *p_out, double *c0_out)
{
    double c0 = x * inv_dx;
    int p = (int)c0;
    if (p > n_g - 2) p = n_g - 2;
    *p_out = p;
    *c0_out = c0;
}

/* The paper's FP64 form: densities in m^-3 (Algorithm 2, including the
 * doubling at the two half-volume edge points). */
void orc_deposit_paper(const double *x, int64_t n, int n_g, double inv_dx, double factor_w, double *dens)
{
    for (int p = 0; p < n_g; ++p) dens[p] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        int p;
        double c0;
        cell_of(x[k], inv_dx, n_g, &p, &c0);
        dens[p] += (p + 1 - c0) * factor_w;
        dens[p + 1] += (c0 - p) * factor_w;
    }
    dens[0] *= 2.0;
    dens[n_g - 1] *= 2.0;
}

/* Fixed-point form: each particle contributes exactly 2^32 units, split as
 * q2 = round-to-nearest-even((c0 - p) * 2^32) to point p+1 and 2^32 - q2 to
 * point p.  Sums are exact integers, so the order of accumulation does not
 * matter.  Densities follow as n_p = FACTOR_W * Q_p / 2^32 (x2 at the edges). */
void orc_deposit_fixed(const double *x, int64_t n, int n_g, double inv_dx, int64_t *q)
{
    for (int p = 0; p < n_g; ++p) q[p] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int p;
        double c0;
        cell_of(x[k], inv_dx, n_g, &p, &c0);
        double c2 = c0 - p;
        int64_t q2 = (int64_t)llrint(c2 * 4294967296.0);
        q[p] += (int64_t)4294967296LL - q2;
        q[p + 1] += q2;
    }
}

/* The same decision taken in FP32 (for the FP32 particle mode: the cell index
 * and split are decided in the precision the particle positions are kept in). */
void orc_deposit_fixed_f32(const float *x, int64_t n, int n_g, float inv_dx, int64_t *q)
{
    for (int p = 0; p < n_g; ++p) q[p] = 0;
    for (int64_t k = 0; k < n; ++k) {
        float c0 = x[k] * inv_dx;
        int p = (int)c0;
        if (p > n_g - 2) p = n_g - 2;
        float c2 = c0 - (float)p;
        int64_t q2 = (int64_t)llrintf(c2 * 4294967296.0f);
        q[p] += (int64_t)4294967296LL - q2;
        q[p + 1] += q2;
    }
}

/* Densities in m^-3 from the fixed-point sums. */
void orc_density_from_fixed(const int64_t *q, int n_g, double factor_w, double *dens)
{
    for (int p = 0; p < n_g; ++p) dens[p] = factor_w * ((double)q[p] * (1.0 / 4294967296.0));
    dens[0] *= 2.0;
    dens[n_g - 1] *= 2.0;
}

/* ------------------------------------------------------------------------ */
/* Step 2 -- potential and field (Sec. 2.1.2, eqs. eq_poisson_discrete,      */
/* eq_efield, eq_efield_b1, eq_efield_b2; Algorithm 3).  The tridiagonal      */
/* system with constant coefficients is solved with the Thomas algorithm.     */
/* Dirichlet conditions: phi_0 = V(t) (powered electrode), phi_{N_G-1} = 0.   */
/* ------------------------------------------------------------------------ */
void orc_poisson(const double *rho, int n_g, double dx, double v_left, double *phi, double *efield)
{
    const double a = -1.0, b = 2.0, c = -1.0; /* sub-, main and super-diagonal */
    int m = n_g - 2;                          /* unknowns phi_1 .. phi_{N_G-2} */
    if (m < 1) return;
    double *cp = (double *)malloc(sizeof(double) * (size_t)m);
    double *dp = (double *)malloc(sizeof(double) * (size_t)m);
    phi[0] = v_left;
    phi[n_g - 1] = 0.0;
    /* forward elimination; the known boundary potentials move to the right-hand side */
    for (int i = 0; i < m; ++i) {
        int p = i + 1;
        double f = dx * dx * rho[p] / ORC_EPSILON0;
        if (p == 1) f -= a * phi[0];
        if (p == n_g - 2) f -= c * phi[n_g - 1];
        if (i == 0) {
            cp[i] = c / b;
            dp[i] = f / b;
        } else {
            double den = b - a * cp[i - 1];
            cp[i] = c / den;
            dp[i] = (f - a * dp[i - 1]) / den;
        }
    }
    /* back substitution */
    phi[m] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i) phi[i + 1] = dp[i] - cp[i] * phi[i + 2];
    /* field at the grid points: central differences inside, one-sided forms with
     * the half-cell charge correction at the electrodes */
    for (int p = 1; p < n_g - 1; ++p) efield[p] = (phi[p - 1] - phi[p + 1]) / (2.0 * dx);
    efield[0] = (phi[0] - phi[1]) / dx - rho[0] * dx / (2.0 * ORC_EPSILON0);
    efield[n_g - 1] = (phi[n_g - 2] - phi[n_g - 1]) / dx + rho[n_g - 1] * dx / (2.0 * ORC_EPSILON0);
    free(cp);
    free(dp);
}

/* Driving voltage at within-cycle step t (Sec. 2; eq. of the reference run
 * V(t) = V0 cos(2 pi f t) and its dual-frequency sum in Sec. 4.2).
 * Reading: the phase is taken from the step index inside the RF cycle, so no
 * time drift accumulates; every drive frequency is a multiple of the cycle
 * frequency (0 gives a DC term). */
static double drive_voltage(const orc_sim *s, int64_t t_in_cycle)
{
    double t = (double)t_in_cycle * s->dt_e;
    double v = 0.0;
    for (int h = 0; h < s->p.n_harm; ++h) v += s->p.harm_volt_v[h] * cos(2.0 * ORC_PI * s->p.harm_freq_hz[h] * t);
    return v + s->v_bias;
}

/* DC self-bias (Sec. 5): a constant voltage added to the powered electrode's
 * potential, from the next field solve on. */
void orc_set_bias(orc_sim *s, double v_bias) { s->v_bias = v_bias; }

/* ------------------------------------------------------------------------ */
/* Step 6 -- collisions (Sec. 2.1.6; Algorithm 6).                            */
/* ------------------------------------------------------------------------ */

/* Post-collision velocity of the projectile (eq. postcoll_velocity1 and the
 * Euler-angle rotation of Sec. 2.1.6): g points along (theta, phi); the new
 * relative velocity has magnitude gp and is deflected by (chi, eta) from g.
 * Inputs are cos/sin of chi and eta.  Output u = unit vector of g'. */
static void deflect(double gx, double gy, double gz, double g, double cc, double sc, double ce, double se,
                    double u[3])
{
    double ct = gx / g;
    /* sin(theta) from the transverse components of g (the definition
     * g = g (cos theta, sin theta cos phi, sin theta sin phi)), which stays
     * accurate when g is nearly along x, where sqrt(1 - cos^2) cancels */
    double st = sqrt(gy * gy + gz * gz) / g;
    double cp, sp;
    if (st == 0.0) { /* Reading: g along x, the azimuth of g is arbitrary */
        cp = 1.0;
        sp = 0.0;
    } else {
        cp = gy / (g * st);
        sp = gz / (g * st);
    }
    u[0] = ct * cc - st * sc * ce;
    u[1] = st * cp * cc + ct * cp * sc * ce - sp * sc * se;
    u[2] = st * sp * cc + ct * sp * sc * ce + cp * sc * se;
}

/* Electron index into a cross-section table (Algorithm 6): nearest bin. */
/* Null-collision method (Sec. 2.1.6, Sec. 5).  Every particle is offered a
 * collision with the constant probability P* = 1 - exp(-nu* dt): picked when
 * its test uniform R < P*.  Reading: the paper picks N P* particles at random;
 * a Bernoulli draw per particle is the parallel form of that choice (the
 * number picked is binomial with mean N P*).  A picked particle collides for
 * real when R' < nu / nu*, otherwise the collision is null.  Reading: R' is
 * R / P*, which given R < P* is uniform on [0, 1) and independent of the
 * pick, so no second random number is drawn.  nu > nu* (an energy past the
 * table) always collides and is counted. */
static int null_real(orc_sim *s, int species, double u, double nu)
{
    s->counters[ORC_C_NULL_TESTED]++;
    if (nu > s->nu_star[species]) s->counters[ORC_C_NULL_OVER]++;
    return u / s->p_star[species] < nu / s->nu_star[species];
}

static int null_collides(orc_sim *s, int species, int64_t k, double nu)
{
    const double u = test_uniform(s->p.seed, k, s->step, species);
    if (!(u < s->p_star[species])) return 0;
    return null_real(s, species, u, nu);
}

static int energy_index(double energy, double de, int n)
{
    double r = energy / de + 0.5;
    if (!(r < (double)n)) return n - 1;
    int k = (int)r;
    return k < n - 1 ? k : n - 1;
}

/* e- + Ar collision (cold gas, v2 = 0).  Process chosen from the partition of
 * [0,1) by sigma_k / sigma_tot (Fig. 7).  Elastic and excitation scatter
 * isotropically; ionisation shares energy by Opal's formula and uses the
 * explicit angles of Sec. 2.1.6.
 * u_proc, u_chi, u_eta, u_opal are uniforms on [0,1).
 * Returns the process (0 elastic, 1 excitation, 2 ionisation) and, for
 * ionisation, the ejected electron velocity in vej[3].
 * Reading: post-collision energies use the COM energy eps_c = mu g^2 / 2; an
 * inelastic process whose COM energy lies below its threshold (possible only
 * through nearest-bin lookup) is executed as elastic and counted. */
int orc_collide_electron(const orc_sim *s, int k, double *vx, double *vy, double *vz, double u_proc, double u_chi,
                         double u_eta, double u_opal, double vej[3], int *subthreshold)
{
    const double m1 = ORC_E_MASS, m2 = s->ar_mass;
    double s0 = s->sigma[0][k], s1 = s->sigma[0][s->cs_n[0] + k], s2 = s->sigma[0][2 * s->cs_n[0] + k];
    double stot = s0 + s1 + s2;
    int proc;
    if (u_proc < s0 / stot)
        proc = 0;
    else if (u_proc < (s0 + s1) / stot)
        proc = 1;
    else
        proc = 2;
    *subthreshold = 0;
    double gx = *vx, gy = *vy, gz = *vz; /* g = v1 - v2 with v2 = 0 */
    double g2 = gx * gx + gy * gy + gz * gz;
    double g = sqrt(g2);
    double wx = (m1 * gx) / (m1 + m2), wy = (m1 * gy) / (m1 + m2), wz = (m1 * gz) / (m1 + m2);
    double eps_c = 0.5 * s->mu_e * g2 / ORC_EV_TO_J;
    if (proc == 1 && eps_c - s->p.e_exc_ev < 0.0) {
        proc = 0;
        *subthreshold = 1;
    }
    if (proc == 2 && eps_c - s->p.e_ion_ev < 0.0) {
        proc = 0;
        *subthreshold = 1;
    }
    double u[3];
    if (proc == 0 || proc == 1) {
        double gp = g;
        if (proc == 1) gp = sqrt(2.0 * (eps_c - s->p.e_exc_ev) * ORC_EV_TO_J / s->mu_e);
        double cc = 1.0 - 2.0 * u_chi; /* chi = arccos(1 - 2 R01) */
        double sc = sqrt(1.0 - cc * cc);
        double eta = 2.0 * ORC_PI * u_eta;
        deflect(gx, gy, gz, g, cc, sc, cos(eta), sin(eta), u);
        double f = m2 / (m1 + m2) * gp;
        *vx = wx + f * u[0];
        *vy = wy + f * u[1];
        *vz = wz + f * u[2];
    } else {
        double avail = eps_c - s->p.e_ion_ev;
        double e_ej = ORC_OPAL_W_EV * tan(u_opal * atan(avail / (2.0 * ORC_OPAL_W_EV)));
        double e_sc = avail - e_ej;
        /* Reading: cos(chi) = sqrt(eps / (eps_c - eps_ion)) for both electrons */
        double cs = sqrt(e_sc / avail), ss = sqrt(1.0 - cs * cs);
        double ce_ = sqrt(e_ej / avail), se_ = sqrt(1.0 - ce_ * ce_);
        double eta = 2.0 * ORC_PI * u_eta; /* eta_e = eta_s + pi */
        double cet = cos(eta), set = sin(eta);
        double gp = sqrt(2.0 * e_sc * ORC_EV_TO_J / s->mu_e);
        deflect(gx, gy, gz, g, cs, ss, cet, set, u);
        double f = m2 / (m1 + m2) * gp;
        *vx = wx + f * u[0];
        *vy = wy + f * u[1];
        *vz = wz + f * u[2];
        /* Reading: the ejected electron leaves along (chi_e, eta_s + pi) with
         * the LAB speed of its energy */
        double ue[3];
        deflect(gx, gy, gz, g, ce_, se_, -cet, -set, ue);
        double vmag = sqrt(2.0 * e_ej * ORC_EV_TO_J / ORC_E_MASS);
        vej[0] = vmag * ue[0];
        vej[1] = vmag * ue[1];
        vej[2] = vmag * ue[2];
    }
    return proc;
}

/* Ar+ + Ar collision with a thermal partner (va).  Isotropic or backward
 * scattering in the COM frame (Sec. 2.1.6 and Sec. 3.2).  Returns 0 for
 * isotropic, 1 for backward. */
int orc_collide_ion(const orc_sim *s, int k, double *vx, double *vy, double *vz, double vax, double vay, double vaz,
                    double u_proc, double u_chi, double u_eta)
{
    const double m1 = s->ar_mass, m2 = s->ar_mass;
    double s0 = s->sigma[1][k], s1 = s->sigma[1][s->cs_n[1] + k];
    double stot = s0 + s1;
    int proc = (u_proc < s0 / stot) ? 0 : 1;
    double gx = *vx - vax, gy = *vy - vay, gz = *vz - vaz;
    double g = sqrt(gx * gx + gy * gy + gz * gz);
    double wx = (m1 * *vx + m2 * vax) / (m1 + m2);
    double wy = (m1 * *vy + m2 * vay) / (m1 + m2);
    double wz = (m1 * *vz + m2 * vaz) / (m1 + m2);
    double cc, sc, ce, se;
    if (proc == 0) {
        cc = 1.0 - 2.0 * u_chi;
        sc = sqrt(1.0 - cc * cc);
        double eta = 2.0 * ORC_PI * u_eta;
        ce = cos(eta);
        se = sin(eta);
    } else { /* chi = pi */
        cc = -1.0;
        sc = 0.0;
        ce = 1.0;
        se = 0.0;
    }
    double u[3];
    deflect(gx, gy, gz, g, cc, sc, ce, se, u);
    double f = m2 / (m1 + m2) * g;
    *vx = wx + f * u[0];
    *vy = wy + f * u[1];
    *vz = wz + f * u[2];
    return proc;
}

/* ------------------------------------------------------------------------ */
/* Simulation object.                                                        */
/* ------------------------------------------------------------------------ */
orc_sim *orc_create(const orc_params *p)
{
    if (p->n_grid < 3 || p->steps_per_cycle < 1 || p->ion_subcycle < 1 || p->n_harm < 0 || p->n_harm > ORC_MAX_HARM ||
        p->capacity < 1 || p->eepf_bins < 1 || p->ifed_bins < 1 || p->xt_bins < 0 ||
        (p->xt_bins > 0 && p->steps_per_cycle % p->xt_bins != 0) || p->sort_every < 0)
        return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    /* Section 3.1 / Table 1 */
    s->dx = p->gap_m / (p->n_grid - 1);
    s->inv_dx = 1.0 / s->dx;
    s->dt_e = 1.0 / (p->cycle_freq_hz * p->steps_per_cycle);
    s->dt_i = p->ion_subcycle * s->dt_e;
    s->factor_w = p->weight / (p->area_m2 * s->dx);
    s->ar_mass = ORC_AR_MASS_U * ORC_AMU;
    s->factor_e = s->dt_e / ORC_E_MASS * ORC_E_CHARGE;
    s->factor_i = s->dt_i / s->ar_mass * ORC_E_CHARGE;
    s->n_gas = p->pressure_pa / (ORC_K_BOLTZMANN * p->gas_temp_k);
    s->mu_e = ORC_E_MASS * s->ar_mass / (ORC_E_MASS + s->ar_mass);
    s->mu_arar = s->ar_mass / 2.0;
    s->sigma_th_ar = sqrt(ORC_K_BOLTZMANN * p->gas_temp_k / s->ar_mass);
    int ng = p->n_grid;
    for (int sp = 0; sp < 2; ++sp) {
        s->sp[sp].x = (double *)calloc((size_t)p->capacity, sizeof(double));
        s->sp[sp].vx = (double *)calloc((size_t)p->capacity, sizeof(double));
        s->sp[sp].vy = (double *)calloc((size_t)p->capacity, sizeof(double));
        s->sp[sp].vz = (double *)calloc((size_t)p->capacity, sizeof(double));
    }
    s->q_e = (int64_t *)calloc((size_t)ng, sizeof(int64_t));
    s->q_i = (int64_t *)calloc((size_t)ng, sizeof(int64_t));
    s->n_e = (double *)calloc((size_t)ng, sizeof(double));
    s->n_i = (double *)calloc((size_t)ng, sizeof(double));
    s->rho = (double *)calloc((size_t)ng, sizeof(double));
    s->phi = (double *)calloc((size_t)ng, sizeof(double));
    s->efield = (double *)calloc((size_t)ng, sizeof(double));
    s->sum_ne = (double *)calloc((size_t)ng, sizeof(double));
    s->sum_ni = (double *)calloc((size_t)ng, sizeof(double));
    s->sum_phi = (double *)calloc((size_t)ng, sizeof(double));
    s->eepf = (int64_t *)calloc((size_t)p->eepf_bins, sizeof(int64_t));
    s->ifed_pow = (int64_t *)calloc((size_t)p->ifed_bins, sizeof(int64_t));
    s->ifed_gnd = (int64_t *)calloc((size_t)p->ifed_bins, sizeof(int64_t));
    s->prod_cap = p->capacity;
    s->prod = (orc_product *)calloc((size_t)s->prod_cap, sizeof(orc_product));
    s->emit = (orc_product *)calloc((size_t)s->prod_cap, sizeof(orc_product));
    s->absorbed = (unsigned char *)calloc((size_t)p->capacity, 1);
    if (p->xt_bins > 0) {
        const size_t m = (size_t)ng * (size_t)p->xt_bins;
        s->nxt = p->xt_bins;
        s->nbin = p->steps_per_cycle / p->xt_bins;
        s->xt_phi = (double *)calloc(m, sizeof(double));
        s->xt_ef = (double *)calloc(m, sizeof(double));
        s->xt_ne = (double *)calloc(m, sizeof(double));
        s->xt_ni = (double *)calloc(m, sizeof(double));
        s->xt_ion = (double *)calloc(m, sizeof(double));
        for (int sp = 0; sp < 2; ++sp) {
            s->xt_wv[sp] = (double *)calloc(m, sizeof(double));
            s->xt_we[sp] = (double *)calloc(m, sizeof(double));
            s->xt_w[sp] = (double *)calloc(m, sizeof(double));
            s->xt_steps[sp] = (int64_t *)calloc((size_t)p->xt_bins, sizeof(int64_t));
        }
    }
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    for (int sp = 0; sp < 2; ++sp) {
        free(s->sp[sp].x);
        free(s->sp[sp].vx);
        free(s->sp[sp].vy);
        free(s->sp[sp].vz);
        free(s->sigma[sp]);
        free(s->sigma_tot[sp]);
    }
    free(s->q_e);
    free(s->q_i);
    free(s->n_e);
    free(s->n_i);
    free(s->rho);
    free(s->phi);
    free(s->efield);
    free(s->sum_ne);
    free(s->sum_ni);
    free(s->sum_phi);
    free(s->xt_phi);
    free(s->xt_ef);
    free(s->xt_ne);
    free(s->xt_ni);
    free(s->xt_ion);
    for (int sp = 0; sp < 2; ++sp) {
        free(s->xt_wv[sp]);
        free(s->xt_we[sp]);
        free(s->xt_w[sp]);
        free(s->xt_steps[sp]);
    }
    free(s->eepf);
    free(s->ifed_pow);
    free(s->ifed_gnd);
    free(s->prod);
    free(s->emit);
    free(s->absorbed);
    free(s);
}

/* Cross-section tables (Section 3.2): sigma[proc][k] at energy k*de (LAB
 * energy for electrons, COM energy for ions); n*sigma_tot is formed here as
 * calc_total_cross_sections() does. */
int orc_set_cross_sections(orc_sim *s, int species, int n_proc, int n_entries, double de_ev, const double *sigma)
{
    if (species < 0 || species > 1 || n_entries < 1 || de_ev <= 0.0) return -1;
    if ((species == 0 && n_proc != 3) || (species == 1 && n_proc != 2)) return -1;
    free(s->sigma[species]);
    free(s->sigma_tot[species]);
    s->cs_n[species] = n_entries;
    s->cs_nproc[species] = n_proc;
    s->cs_de[species] = de_ev;
    s->sigma[species] = (double *)malloc(sizeof(double) * (size_t)n_proc * (size_t)n_entries);
    memcpy(s->sigma[species], sigma, sizeof(double) * (size_t)n_proc * (size_t)n_entries);
    s->sigma_tot[species] = (double *)malloc(sizeof(double) * (size_t)n_entries);
    for (int k = 0; k < n_entries; ++k) {
        double t = 0.0;
        for (int j = 0; j < n_proc; ++j) t += sigma[(size_t)j * n_entries + k];
        s->sigma_tot[species][k] = t * s->n_gas;
    }
    /* Null-collision bound (Sec. 2.1.6): nu* = max over the table of
     * n sigma_tot v.  Energies round to the nearest entry, so entry k serves
     * energies below (k + 1/2) de, and v is taken there (electrons: lab speed;
     * ions: relative speed with the reduced mass, as the tables are indexed
     * by centre-of-mass energy).  Only energies past the table can exceed it. */
    {
        const double m = species == 0 ? ORC_E_MASS : s->mu_arar;
        double best = 0.0;
        for (int k = 0; k < n_entries; ++k) {
            const double v = sqrt(2.0 * ((k + 0.5) * de_ev) * ORC_EV_TO_J / m);
            const double nu = s->sigma_tot[species][k] * v;
            if (nu > best) best = nu;
        }
        s->nu_star[species] = best;
        s->p_star[species] = 1.0 - exp(-best * (species == 0 ? s->dt_e : s->dt_i));
    }
    return 0;
}

int orc_load_particles(orc_sim *s, int species, int64_t n, const double *x, const double *vx, const double *vy,
                       const double *vz)
{
    if (species < 0 || species > 1 || n < 0 || n > s->p.capacity) return -1;
    orc_species *sp = &s->sp[species];
    sp->n = n;
    memcpy(sp->x, x, sizeof(double) * (size_t)n);
    memcpy(sp->vx, vx, sizeof(double) * (size_t)n);
    memcpy(sp->vy, vy, sizeof(double) * (size_t)n);
    memcpy(sp->vz, vz, sizeof(double) * (size_t)n);
    /* Reading (Algorithms 1-2): a loaded species replaces its deposited
     * density at once, also between ion steps when the ion density is held. */
    orc_deposit_fixed(sp->x, n, s->p.n_grid, s->inv_dx, species == 0 ? s->q_e : s->q_i);
    return 0;
}

/* Initialisation of Algorithm 1, init(N_INIT): n electrons and n Ar+ at
 * random positions in the gap with zero velocities.  Reading: particle k of
 * species s sits at x = L R01 with R01 from block 9 of its counter (slot k,
 * the current step), so that the seeding is reproducible in any order. */
int orc_seed(orc_sim *s, int64_t n)
{
    if (n < 0 || n > s->p.capacity) return -1;
    for (int species = 0; species < 2; ++species) {
        orc_species *sp = &s->sp[species];
        for (int64_t k = 0; k < n; ++k) {
            double u[2];
            draw_block(s->p.seed, k, s->step, species, 9, u);
            sp->x[k] = s->p.gap_m * u[0];
            sp->vx[k] = sp->vy[k] = sp->vz[k] = 0.0;
        }
        sp->n = n;
        orc_deposit_fixed(sp->x, n, s->p.n_grid, s->inv_dx, species == 0 ? s->q_e : s->q_i);
    }
    return 0;
}

/* Steps (1)-(2) of the current step without advancing it: the densities and
 * the field that the next call of one_step() will use. */
void orc_prepare_fields(orc_sim *s)
{
    const int ng = s->p.n_grid;
    const int64_t t = s->step % s->p.steps_per_cycle;
    orc_deposit_fixed(s->sp[ORC_SPECIES_E].x, s->sp[ORC_SPECIES_E].n, ng, s->inv_dx, s->q_e);
    if ((t % s->p.ion_subcycle) == 0) orc_deposit_fixed(s->sp[ORC_SPECIES_I].x, s->sp[ORC_SPECIES_I].n, ng, s->inv_dx, s->q_i);
    orc_density_from_fixed(s->q_e, ng, s->factor_w, s->n_e);
    orc_density_from_fixed(s->q_i, ng, s->factor_w, s->n_i);
    for (int k = 0; k < ng; ++k) s->rho[k] = ORC_E_CHARGE * (s->n_i[k] - s->n_e[k]);
    orc_poisson(s->rho, ng, s->dx, drive_voltage(s, t), s->phi, s->efield);
}

int64_t orc_count(const orc_sim *s, int species) { return s->sp[species].n; }

int orc_get_particles(const orc_sim *s, int species, double *x, double *vx, double *vy, double *vz)
{
    const orc_species *sp = &s->sp[species];
    memcpy(x, sp->x, sizeof(double) * (size_t)sp->n);
    memcpy(vx, sp->vx, sizeof(double) * (size_t)sp->n);
    memcpy(vy, sp->vy, sizeof(double) * (size_t)sp->n);
    memcpy(vz, sp->vz, sizeof(double) * (size_t)sp->n);
    return 0;
}

/* Canonical removal (step 5) and append: holes below the new count are filled,
 * in ascending order, by the surviving particles of the tail [N', N) in
 * ascending order; created particles are then appended in ascending order of
 * their parent's slot.  Reading: the paper's swap-with-last loop (Algorithm 5)
 * leaves the same set of particles in another order; this order is the one
 * used for per-slot comparison. */
static void compact(orc_species *sp, const unsigned char *absorbed)
{
    int64_t n = sp->n, holes = 0;
    for (int64_t j = 0; j < n; ++j) holes += absorbed[j];
    int64_t nn = n - holes;
    int64_t src = nn;
    for (int64_t j = 0; j < nn; ++j) {
        if (!absorbed[j]) continue;
        while (absorbed[src]) ++src;
        sp->x[j] = sp->x[src];
        sp->vx[j] = sp->vx[src];
        sp->vy[j] = sp->vy[src];
        sp->vz[j] = sp->vz[src];
        ++src;
    }
    sp->n = nn;
}

/* Periodic cell sort (not part of the paper's method; the GPU build keeps
 * particles of a cell together so that its block-local deposition and field
 * gathers touch few cells).  Reading: after a step whose new index s is a
 * multiple of sort_every * N_SUB, the particles of each species are put in
 * ascending order of their cell p (the cell of the deposition, Algorithm 2),
 * keeping the order of the slots within a cell (a stable sort).  The slot of
 * a particle, and with it the counter of its random numbers, follows the new
 * order.  A counting sort: the cell histogram, its exclusive prefix sum as
 * the first slot of each cell, then one pass in slot order. */
static void sort_species(orc_sim *s, orc_species *sp)
{
    const int ng = s->p.n_grid;
    const int64_t n = sp->n;
    if (n < 2) return;
    int64_t *first = (int64_t *)calloc((size_t)ng, sizeof(int64_t));
    int *cellv = (int *)malloc(sizeof(int) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        int c;
        double c0;
        cell_of(sp->x[j], s->inv_dx, ng, &c, &c0);
        cellv[j] = c;
        first[c] += 1;
    }
    int64_t run = 0;
    for (int c = 0; c < ng; ++c) {
        const int64_t h = first[c];
        first[c] = run;
        run += h;
    }
    double *a[4] = {sp->x, sp->vx, sp->vy, sp->vz};
    for (int k = 0; k < 4; ++k) {
        double *out = (double *)malloc(sizeof(double) * (size_t)n);
        int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)ng);
        memcpy(next, first, sizeof(int64_t) * (size_t)ng);
        for (int64_t j = 0; j < n; ++j) out[next[cellv[j]]++] = a[k][j];
        memcpy(a[k], out, sizeof(double) * (size_t)n);
        free(out);
        free(next);
    }
    free(first);
    free(cellv);
}

/* Adds (c1 a, c2 a) to grid points (c, c+1) of time bin b of an xt array
 * (the weights of the density assignment, Sec. 2.1.1). */
static void xt_add(const orc_sim *s, double *xt, double x, int b, double a)
{
    int c;
    double c0;
    cell_of(x, s->inv_dx, s->p.n_grid, &c, &c0);
    xt[(size_t)c * s->nxt + b] += (c + 1 - c0) * a;
    xt[(size_t)(c + 1) * s->nxt + b] += (c0 - c) * a;
}

/* One particle's contribution to the xt sums of its species: at x(t), with
 * the time-centred velocity v_c (Sec. 3.5). */
static void xt_particle(const orc_sim *s, int species, double x, double vcx, double vy, double vz, int b)
{
    const double m = species == ORC_SPECIES_E ? ORC_E_MASS : s->ar_mass;
    const double en = 0.5 * m * (vcx * vcx + vy * vy + vz * vz) / ORC_EV_TO_J;
    xt_add(s, s->xt_wv[species], x, b, vcx);
    xt_add(s, s->xt_we[species], x, b, en);
    xt_add(s, s->xt_w[species], x, b, 1.0);
}

/* One PIC/MCC time step (Sec. 2.1, Fig. 2; Algorithms 2-6). */
static void one_step(orc_sim *s, int measure)
{
    const orc_params *p = &s->p;
    const int ng = p->n_grid;
    const int64_t t = s->step % p->steps_per_cycle; /* within-cycle step */
    const int ion_step = (t % p->ion_subcycle) == 0;
    orc_species *E = &s->sp[ORC_SPECIES_E], *I = &s->sp[ORC_SPECIES_I];
    const int xt_on = measure && s->nxt > 0;
    const int xb = s->nxt > 0 ? (int)(t / s->nbin) : 0; /* time bin of this step */

    /* (1) densities (Algorithm 2), every step for e-, every N_SUB-th for Ar+.
     * Reading: the densities are reset before every deposition. */
    orc_deposit_fixed(E->x, E->n, ng, s->inv_dx, s->q_e);
    if (ion_step) orc_deposit_fixed(I->x, I->n, ng, s->inv_dx, s->q_i);
    orc_density_from_fixed(s->q_e, ng, s->factor_w, s->n_e);
    orc_density_from_fixed(s->q_i, ng, s->factor_w, s->n_i);

    /* (2) rho, potential and field (Algorithm 3) */
    for (int k = 0; k < ng; ++k) s->rho[k] = ORC_E_CHARGE * (s->n_i[k] - s->n_e[k]);
    orc_poisson(s->rho, ng, s->dx, drive_voltage(s, t), s->phi, s->efield);

    /* (3,4) field at the particles and leapfrog push (Algorithm 4);
     * EEPF sampled in the centre 10% of the gap with the time-centred velocity
     * (Sec. 3.5).  Reading: the sample uses x(t) and v(t) = (v(t-dt/2) +
     * v(t+dt/2))/2. */
    s->counters[ORC_C_PUSH_E] += E->n;
    if (ion_step) s->counters[ORC_C_PUSH_I] += I->n;
    for (int64_t k = 0; k < E->n; ++k) {
        int c;
        double c0;
        cell_of(E->x[k], s->inv_dx, ng, &c, &c0);
        double c1 = c + 1 - c0, c2 = c0 - c;
        double e_x = c1 * s->efield[c] + c2 * s->efield[c + 1];
        double vx_old = E->vx[k];
        E->vx[k] -= e_x * s->factor_e;
        if (measure) {
            /* power absorption (Sec. 3.5): the field's work on the particle
             * over the step, q E_x v_c dt with the time-centred velocity */
            s->work[ORC_SPECIES_E] += -ORC_E_CHARGE * e_x * (0.5 * (vx_old + E->vx[k])) * s->dt_e;
            double xo = E->x[k];
            if (xo >= 0.45 * p->gap_m && xo <= 0.55 * p->gap_m) {
                double vc = 0.5 * (vx_old + E->vx[k]);
                double v2 = vc * vc + E->vy[k] * E->vy[k] + E->vz[k] * E->vz[k];
                double en = 0.5 * ORC_E_MASS * v2 / ORC_EV_TO_J;
                double r = en / p->eepf_de_ev;
                if (r < (double)p->eepf_bins) s->eepf[(int)r] += 1;
            }
            if (xt_on) xt_particle(s, ORC_SPECIES_E, xo, 0.5 * (vx_old + E->vx[k]), E->vy[k], E->vz[k], xb);
        }
        E->x[k] += E->vx[k] * s->dt_e;
    }
    if (ion_step) {
        for (int64_t k = 0; k < I->n; ++k) {
            int c;
            double c0;
            cell_of(I->x[k], s->inv_dx, ng, &c, &c0);
            double c1 = c + 1 - c0, c2 = c0 - c;
            double e_x = c1 * s->efield[c] + c2 * s->efield[c + 1];
            double vx_old = I->vx[k];
            I->vx[k] += e_x * s->factor_i;
            if (measure) s->work[ORC_SPECIES_I] += ORC_E_CHARGE * e_x * (0.5 * (vx_old + I->vx[k])) * s->dt_i;
            if (xt_on) xt_particle(s, ORC_SPECIES_I, I->x[k], 0.5 * (vx_old + I->vx[k]), I->vy[k], I->vz[k], xb);
            I->x[k] += I->vx[k] * s->dt_i;
        }
    }

    /* (5) absorption at the electrodes (Algorithm 5): x < 0 at the powered
     * electrode, x > L at the grounded one.  Ar+ energies at impact build the
     * IFEDF (Sec. 3.5).  Surface process (Sec. 5): an electron reaching
     * electrode s is reflected elastically when R01 < eta_s (block 5).
     * Reading: the reflection mirrors the particle back into the gap (x ->
     * -x, or 2L - x) and reverses v_x; if the mirror image is still outside
     * the gap, the electron is absorbed. */
    for (int64_t k = 0; k < E->n; ++k) {
        unsigned char out = 0;
        const double x = E->x[k];
        if (x < 0.0 || x > p->gap_m) {
            const int side = x < 0.0 ? 0 : 1;
            int reflected = 0;
            if (p->refl_eta[side] > 0.0) {
                double u[2];
                draw_block(p->seed, k, s->step, ORC_SPECIES_E, 5, u);
                const double xr = side == 0 ? -x : 2.0 * p->gap_m - x;
                if (u[0] < p->refl_eta[side] && xr >= 0.0 && xr <= p->gap_m) {
                    E->x[k] = xr;
                    E->vx[k] = -E->vx[k];
                    s->counters[ORC_C_REFLECTED]++;
                    reflected = 1;
                }
            }
            if (!reflected) {
                s->counters[ORC_C_ABS_E_POW + side]++;
                out = 1;
            }
        }
        s->absorbed[k] = out;
    }

    /* (6) e- collisions (Algorithm 6), for the particles still in the gap, in
     * slot order; random numbers keyed by (slot, step). */
    int64_t nprod = 0;
    for (int64_t k = 0; k < E->n; ++k) {
        if (s->absorbed[k]) continue;
        double v2 = E->vx[k] * E->vx[k] + E->vy[k] * E->vy[k] + E->vz[k] * E->vz[k];
        double velocity = sqrt(v2);
        double energy = 0.5 * ORC_E_MASS * v2 / ORC_EV_TO_J;
        int ei = energy_index(energy, s->cs_de[0], s->cs_n[0]);
        double nu = s->sigma_tot[0][ei] * velocity;
        if ((p->null_collision & 1) ? null_collides(s, 0, k, nu)
                              : test_uniform(p->seed, k, s->step, ORC_SPECIES_E) < 1.0 - exp(-nu * s->dt_e)) {
            /* Reading: a collision happens when R01 < P_coll (Algorithm 6) */
            double ua[2], ub[2], vej[3];
            int sub;
            draw_block(p->seed, k, s->step, ORC_SPECIES_E, 1, ua);
            draw_block(p->seed, k, s->step, ORC_SPECIES_E, 2, ub);
            int proc = orc_collide_electron(s, ei, &E->vx[k], &E->vy[k], &E->vz[k], ua[0], ua[1], ub[0], ub[1], vej,
                                            &sub);
            s->counters[ORC_C_COLL_E_ELA + proc]++;
            s->counters[ORC_C_SUBTHRESHOLD] += sub;
            if (proc == 2) {
                /* ionisation rate map: the event at the collision position */
                if (xt_on) xt_add(s, s->xt_ion, E->x[k], xb, 1.0);
                /* Reading: the new Ar+ is drawn from the gas Maxwellian */
                double n1[2], n2[2], z1[2], z2[2];
                draw_block(p->seed, k, s->step, ORC_SPECIES_E, 3, n1);
                draw_block(p->seed, k, s->step, ORC_SPECIES_E, 4, n2);
                box_muller(n1, z1);
                box_muller(n2, z2);
                orc_product *pr = &s->prod[nprod++];
                pr->parent = k;
                pr->x = E->x[k];
                pr->vxe = vej[0];
                pr->vye = vej[1];
                pr->vze = vej[2];
                pr->vxi = s->sigma_th_ar * z1[0];
                pr->vyi = s->sigma_th_ar * z1[1];
                pr->vzi = s->sigma_th_ar * z2[0];
            }
        }
    }
    compact(E, s->absorbed);

    int64_t nemit = 0;
    if (ion_step) {
        for (int64_t k = 0; k < I->n; ++k) {
            unsigned char out = 0;
            double en = -1.0;
            /* Surface process (Sec. 5): an ion reaching electrode s emits an
             * electron when R01 < gamma_s (block 5).  Reading: the electron
             * starts at the electrode with a half-Maxwellian velocity at
             * see_te_ev pointing into the gap (blocks 6, 7). */
            if ((I->x[k] < 0.0 || I->x[k] > p->gap_m) && p->see_gamma[I->x[k] < 0.0 ? 0 : 1] > 0.0) {
                const int side = I->x[k] < 0.0 ? 0 : 1;
                double u[2];
                draw_block(p->seed, k, s->step, ORC_SPECIES_I, 5, u);
                if (u[0] < p->see_gamma[side]) {
                    double a[2], b[2], za[2], zb[2];
                    draw_block(p->seed, k, s->step, ORC_SPECIES_I, 6, a);
                    draw_block(p->seed, k, s->step, ORC_SPECIES_I, 7, b);
                    box_muller(a, za);
                    box_muller(b, zb);
                    const double sth = sqrt(p->see_te_ev * ORC_EV_TO_J / ORC_E_MASS);
                    s->counters[ORC_C_EMITTED_POW + side]++;
                    orc_product *em = &s->emit[nemit++];
                    em->parent = k;
                    em->x = side == 0 ? 0.0 : p->gap_m;
                    em->vxe = (side == 0 ? 1.0 : -1.0) * sth * fabs(za[0]);
                    em->vye = sth * za[1];
                    em->vze = sth * zb[0];
                }
            }
            if (I->x[k] < 0.0 || I->x[k] > p->gap_m) {
                double v2 = I->vx[k] * I->vx[k] + I->vy[k] * I->vy[k] + I->vz[k] * I->vz[k];
                en = 0.5 * s->ar_mass * v2 / ORC_EV_TO_J;
            }
            if (I->x[k] < 0.0) {
                s->counters[ORC_C_ABS_I_POW]++;
                out = 1;
                if (measure) {
                    double r = en / p->ifed_de_ev;
                    if (r < (double)p->ifed_bins) s->ifed_pow[(int)r] += 1;
                }
            }
            if (I->x[k] > p->gap_m) {
                s->counters[ORC_C_ABS_I_GND]++;
                out = 1;
                if (measure) {
                    double r = en / p->ifed_de_ev;
                    if (r < (double)p->ifed_bins) s->ifed_gnd[(int)r] += 1;
                }
            }
            s->absorbed[k] = out;
        }
        /* Ar+ collisions with a thermal partner drawn before P_coll */
        for (int64_t k = 0; k < I->n; ++k) {
            if (s->absorbed[k]) continue;
            /* null-collision method: only the P* share of the ions draws a partner */
            const double u_test = test_uniform(p->seed, k, s->step, ORC_SPECIES_I);
            if ((p->null_collision & 2) && !(u_test < s->p_star[1])) continue;
            double ua[2], ub[2], za[2], zb[2], uc[2], ud[2];
            draw_block(p->seed, k, s->step, ORC_SPECIES_I, 1, ua);
            draw_block(p->seed, k, s->step, ORC_SPECIES_I, 2, ub);
            box_muller(ua, za);
            box_muller(ub, zb);
            double vx_a = s->sigma_th_ar * za[0], vy_a = s->sigma_th_ar * za[1], vz_a = s->sigma_th_ar * zb[0];
            double gx = I->vx[k] - vx_a, gy = I->vy[k] - vy_a, gz = I->vz[k] - vz_a;
            double g_sqr = gx * gx + gy * gy + gz * gz;
            double g = sqrt(g_sqr);
            double energy = 0.5 * s->mu_arar * g_sqr / ORC_EV_TO_J;
            int ei = energy_index(energy, s->cs_de[1], s->cs_n[1]);
            double nu = s->sigma_tot[1][ei] * g;
            if ((p->null_collision & 2) ? null_real(s, 1, u_test, nu) : u_test < 1.0 - exp(-nu * s->dt_i)) {
                draw_block(p->seed, k, s->step, ORC_SPECIES_I, 3, uc);
                draw_block(p->seed, k, s->step, ORC_SPECIES_I, 4, ud);
                int proc = orc_collide_ion(s, ei, &I->vx[k], &I->vy[k], &I->vz[k], vx_a, vy_a, vz_a, uc[0], uc[1],
                                           ud[0]);
                s->counters[ORC_C_COLL_I_ISO + proc]++;
            }
        }
        compact(I, s->absorbed);
    }

    /* created pairs join the arrays, in ascending parent order (the loop above
     * already visits parents in ascending order) */
    for (int64_t j = 0; j < nprod; ++j) {
        const orc_product *pr = &s->prod[j];
        if (E->n >= p->capacity || I->n >= p->capacity) {
            s->counters[ORC_C_DROPPED]++;
            s->error = 1;
            continue;
        }
        E->x[E->n] = pr->x;
        E->vx[E->n] = pr->vxe;
        E->vy[E->n] = pr->vye;
        E->vz[E->n] = pr->vze;
        E->n++;
        I->x[I->n] = pr->x;
        I->vx[I->n] = pr->vxi;
        I->vy[I->n] = pr->vyi;
        I->vz[I->n] = pr->vzi;
        I->n++;
        s->counters[ORC_C_CREATED]++;
    }
    /* then the secondary electrons, in ascending order of the emitting ion */
    for (int64_t j = 0; j < nemit; ++j) {
        const orc_product *em = &s->emit[j];
        if (E->n >= p->capacity) {
            s->counters[ORC_C_DROPPED]++;
            s->error = 1;
            continue;
        }
        E->x[E->n] = em->x;
        E->vx[E->n] = em->vxe;
        E->vy[E->n] = em->vye;
        E->vz[E->n] = em->vze;
        E->n++;
    }

    /* grid diagnostics of this step (Sec. 3.6: accumulated after the six steps) */
    if (measure) {
        for (int k = 0; k < ng; ++k) {
            s->sum_ne[k] += s->n_e[k];
            s->sum_ni[k] += s->n_i[k];
            s->sum_phi[k] += s->phi[k];
        }
        s->measured_steps++;
    }
    if (xt_on) {
        for (int k = 0; k < ng; ++k) {
            const size_t j = (size_t)k * s->nxt + xb;
            s->xt_phi[j] += s->phi[k];
            s->xt_ef[j] += s->efield[k];
            s->xt_ne[j] += s->n_e[k];
            s->xt_ni[j] += s->n_i[k];
        }
        s->xt_steps[0][xb]++;
        if (ion_step) s->xt_steps[1][xb]++;
    }
    s->step++;
    if (p->sort_every > 0 && s->step % ((int64_t)p->sort_every * p->ion_subcycle) == 0) {
        sort_species(s, E);
        sort_species(s, I);
    }
}

int orc_step(orc_sim *s, int64_t n_steps, int measure)
{
    if (!s->sigma[0] || !s->sigma[1]) return -1;
    for (int64_t i = 0; i < n_steps; ++i) one_step(s, measure);
    return s->error ? -2 : 0;
}

int64_t orc_get_step(const orc_sim *s) { return s->step; }
void orc_set_step(orc_sim *s, int64_t step) { s->step = step; }

/* Fields of the last step: densities, rho, phi, E, and the fixed-point sums. */
void orc_get_fields(const orc_sim *s, double *ne, double *ni, double *phi, double *efield, int64_t *qe, int64_t *qi)
{
    int ng = s->p.n_grid;
    if (ne) memcpy(ne, s->n_e, sizeof(double) * (size_t)ng);
    if (ni) memcpy(ni, s->n_i, sizeof(double) * (size_t)ng);
    if (phi) memcpy(phi, s->phi, sizeof(double) * (size_t)ng);
    if (efield) memcpy(efield, s->efield, sizeof(double) * (size_t)ng);
    if (qe) memcpy(qe, s->q_e, sizeof(int64_t) * (size_t)ng);
    if (qi) memcpy(qi, s->q_i, sizeof(int64_t) * (size_t)ng);
}

void orc_get_counters(const orc_sim *s, int64_t out[19]) { memcpy(out, s->counters, sizeof(s->counters)); }

/* Time-averaged diagnostics (Sec. 3.5): densities and potential averaged over
 * the measured steps; EEPF normalised to sum f sqrt(eps) dE = 1 at bin centres;
 * IFEDF normalised to sum F dE = 1. */
int64_t orc_get_diagnostics(const orc_sim *s, double *ne_avg, double *ni_avg, double *phi_avg, int64_t *eepf_counts,
                            int64_t *ifed_pow_counts, int64_t *ifed_gnd_counts)
{
    int ng = s->p.n_grid;
    double m = s->measured_steps > 0 ? (double)s->measured_steps : 1.0;
    for (int k = 0; k < ng; ++k) {
        if (ne_avg) ne_avg[k] = s->sum_ne[k] / m;
        if (ni_avg) ni_avg[k] = s->sum_ni[k] / m;
        if (phi_avg) phi_avg[k] = s->sum_phi[k] / m;
    }
    if (eepf_counts) memcpy(eepf_counts, s->eepf, sizeof(int64_t) * (size_t)s->p.eepf_bins);
    if (ifed_pow_counts) memcpy(ifed_pow_counts, s->ifed_pow, sizeof(int64_t) * (size_t)s->p.ifed_bins);
    if (ifed_gnd_counts) memcpy(ifed_gnd_counts, s->ifed_gnd, sizeof(int64_t) * (size_t)s->p.ifed_bins);
    return s->measured_steps;
}

/* Power absorption by e- and Ar+ (Sec. 3.5): the space and time average of
 * j E over the gap and the measured time, = (work per unit weight) W /
 * (A L T_meas), with T_meas = measured steps x dt_e.  W/m^3. */
int64_t orc_get_power(const orc_sim *s, double out[2])
{
    const double t = (double)s->measured_steps * s->dt_e;
    for (int k = 0; k < 2; ++k)
        out[k] = t > 0.0 ? s->work[k] * s->p.weight / (s->p.area_m2 * s->p.gap_m * t) : 0.0;
    return s->measured_steps;
}

void orc_eepf_normalise(const int64_t *h, int n, double de, double *energy, double *f)
{
    double tot = 0.0;
    for (int k = 0; k < n; ++k) tot += (double)h[k];
    for (int k = 0; k < n; ++k) {
        energy[k] = (k + 0.5) * de;
        f[k] = tot > 0.0 ? (double)h[k] / (tot * de * sqrt(energy[k])) : 0.0;
    }
}

void orc_ifed_normalise(const int64_t *h, int n, double de, double *energy, double *f)
{
    double tot = 0.0;
    for (int k = 0; k < n; ++k) tot += (double)h[k];
    for (int k = 0; k < n; ++k) {
        energy[k] = (k + 0.5) * de;
        f[k] = tot > 0.0 ? (double)h[k] / (tot * de) : 0.0;
    }
}

/* Derived quantities, for tests. */
/* The xt map of quantity q (0 phi, 1 E, 2 n_e, 3 n_i, 4 j_e, 5 j_i, 6 power
 * e-, 7 power Ar+, 8 mean e- energy, 9 mean Ar+ energy, 10 ionisation rate),
 * [n_grid][xt_bins], averaged over the measured steps of each bin (ions: the
 * ion steps).  Readings: j = q FACTOR_W sum(w v_c,x) per step, with the
 * density's doubling at the two half-volume edge points; the power map is the
 * product j E of the current and field maps (Sec. 3.5 describes the power as
 * the average of j E and its xt file as that product); the mean energies are
 * in eV; the ionisation rate is FACTOR_W sum(w) per step (doubled at the
 * edges) over dt_e.  Returns -1 without xt diagnostics. */
int orc_get_xt(const orc_sim *s, int q, double *out)
{
    if (s->nxt < 1 || q < 0 || q > 10) return -1;
    const int ng = s->p.n_grid, nxt = s->nxt;
    for (int k = 0; k < ng; ++k) {
        const double edge = (k == 0 || k == ng - 1) ? 2.0 : 1.0;
        for (int b = 0; b < nxt; ++b) {
            const size_t j = (size_t)k * nxt + b;
            const double n0 = (double)s->xt_steps[0][b], n1 = (double)s->xt_steps[1][b];
            const double je = n0 > 0 ? -ORC_E_CHARGE * s->factor_w * edge * s->xt_wv[0][j] / n0 : 0.0;
            const double ji = n1 > 0 ? ORC_E_CHARGE * s->factor_w * edge * s->xt_wv[1][j] / n1 : 0.0;
            const double ef = n0 > 0 ? s->xt_ef[j] / n0 : 0.0;
            double v = 0.0;
            switch (q) {
                case 0: v = n0 > 0 ? s->xt_phi[j] / n0 : 0.0; break;
                case 1: v = ef; break;
                case 2: v = n0 > 0 ? s->xt_ne[j] / n0 : 0.0; break;
                case 3: v = n0 > 0 ? s->xt_ni[j] / n0 : 0.0; break;
                case 4: v = je; break;
                case 5: v = ji; break;
                case 6: v = je * ef; break;
                case 7: v = ji * ef; break;
                case 8: v = s->xt_w[0][j] > 0 ? s->xt_we[0][j] / s->xt_w[0][j] : 0.0; break;
                case 9: v = s->xt_w[1][j] > 0 ? s->xt_we[1][j] / s->xt_w[1][j] : 0.0; break;
                default: v = n0 > 0 ? s->factor_w * edge * s->xt_ion[j] / (n0 * s->dt_e) : 0.0; break;
            }
            out[j] = v;
        }
    }
    return 0;
}

void orc_get_derived(const orc_sim *s, double out[16])
{
    out[12] = s->nu_star[0];
    out[13] = s->nu_star[1];
    out[14] = s->p_star[0];
    out[15] = s->p_star[1];
    out[0] = s->dx;
    out[1] = s->inv_dx;
    out[2] = s->dt_e;
    out[3] = s->dt_i;
    out[4] = s->factor_w;
    out[5] = s->factor_e;
    out[6] = s->factor_i;
    out[7] = s->n_gas;
    out[8] = s->ar_mass;
    out[9] = s->mu_e;
    out[10] = s->mu_arar;
    out[11] = s->sigma_th_ar;
}

/* Unit entry points for the collision pins: one collision with given random
 * numbers, using the loaded cross sections. */
int orc_unit_collide_electron(orc_sim *s, int k, double v[3], double u_proc, double u_chi, double u_eta, double u_opal,
                              double vej[3])
{
    int sub;
    return orc_collide_electron(s, k, &v[0], &v[1], &v[2], u_proc, u_chi, u_eta, u_opal, vej, &sub);
}

int orc_unit_collide_ion(orc_sim *s, int k, double v[3], const double va[3], double u_proc, double u_chi, double u_eta)
{
    return orc_collide_ion(s, k, &v[0], &v[1], &v[2], va[0], va[1], va[2], u_proc, u_chi, u_eta);
}

/* FP32 process selection (the decision taken in the FP32 particle mode's
 * precision): thresholds are the FP64 cumulative fractions rounded to float. */
int orc_select_process_f32(const orc_sim *s, int species, int k, float u)
{
    int n = s->cs_n[species];
    if (species == 0) {
        double s0 = s->sigma[0][k], s1 = s->sigma[0][n + k], s2 = s->sigma[0][2 * n + k];
        double stot = s0 + s1 + s2;
        float t1 = (float)(s0 / stot), t2 = (float)((s0 + s1) / stot);
        return u < t1 ? 0 : (u < t2 ? 1 : 2);
    }
    double s0 = s->sigma[1][k], s1 = s->sigma[1][n + k];
    float t1 = (float)(s0 / (s0 + s1));
    return u < t1 ? 0 : 1;
}

/* FP64 process selection, as used inside orc_collide_electron/ion. */
int orc_select_process(const orc_sim *s, int species, int k, double u)
{
    int n = s->cs_n[species];
    if (species == 0) {
        double s0 = s->sigma[0][k], s1 = s->sigma[0][n + k], s2 = s->sigma[0][2 * n + k];
        double stot = s0 + s1 + s2;
        return u < s0 / stot ? 0 : (u < (s0 + s1) / stot ? 1 : 2);
    }
    double s0 = s->sigma[1][k], s1 = s->sigma[1][n + k];
    return u < s0 / (s0 + s1) ? 0 : 1;
}
