/*
 * edupic.h -- C ABI of the GB300 (sm_103a) PIC/MCC particle-loop library.
 *
 * The library steps one or more independent 1D3V electrostatic PIC/MCC
 * simulations of argon capacitively coupled plasmas (Donko et al., arXiv
 * 2103.09642): leapfrog push (Sec. 2.1.4, Algorithm 4), linear-weighting
 * deposition (Sec. 2.1.1, Algorithm 2), electrode absorption with compaction
 * (Sec. 2.1.5, Algorithm 5), e- + Ar and Ar+ + Ar Monte Carlo collisions
 * (Sec. 2.1.6, Algorithm 6) with ion subcycling (Sec. 2.1), around a 1D
 * Poisson solve (Sec. 2.1.2, Algorithm 3).  Every step runs in hand-written
 * CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Return EDUPIC_OK (0) on success or a negative EDUPIC_E* status.
 *  - Pointers documented as "host" are host memory owned by the caller and
 *    only read/written during the call.  Pointers documented as "device" are
 *    CUDA device memory owned by the caller.
 *  - Work is enqueued on the stream given at creation.  Calls that return
 *    host data synchronise that stream first; edupic_step / edupic_run_cycles
 *    only enqueue.  Errors found on the device (capacity overflow, non-finite
 *    particle data) are reported by the next synchronising call.
 *  - A simulation object is not thread-safe.  Distinct objects may be used
 *    from distinct threads on distinct streams.
 */
#ifndef EDUPIC_H
#define EDUPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define EDUPIC_OK 0
#define EDUPIC_EINVAL (-1)    /* invalid argument or parameter set */
#define EDUPIC_ENOMEM (-2)    /* arena too small / HBM budget exceeded */
#define EDUPIC_ECAPACITY (-3) /* particle, hole or product capacity exceeded */
#define EDUPIC_ECUDA (-4)     /* a CUDA runtime call failed */
#define EDUPIC_ESTATE (-5)    /* call not valid in the current state */
#define EDUPIC_ENAN (-6)      /* non-finite particle position found */
#define EDUPIC_EIO (-7)       /* checkpoint file could not be read/written */
#define EDUPIC_ETIMEOUT (-8)  /* bounded wait expired */
#define EDUPIC_ETOOBIG (-9)   /* size beyond the fixed scratch of edupic_fields_noalloc */
#define EDUPIC_ESTABILITY (-10) /* an accuracy/stability condition fails (edupic_check_accuracy) */

/* ---------------------------------------------------------------- enums */
#define EDUPIC_FP64 0 /* particles, push and collisions in FP64 */
#define EDUPIC_FP32 1 /* particles, push and collisions in FP32; field and diagnostics FP64 */

#define EDUPIC_ELECTRONS 0
#define EDUPIC_IONS 1

#define EDUPIC_MAX_HARMONICS 4
#define EDUPIC_MAX_GRID 2048       /* largest N_G */
#define EDUPIC_MAX_EEPF_BINS 2048
#define EDUPIC_MAX_IFED_BINS 4096
#define EDUPIC_MAX_DISCHARGES 1024 /* discharges per simulation object */
#define EDUPIC_MAX_CS_ENTRIES 4194304 /* cross-section table length (2^22) */
#define EDUPIC_STEP_EVENTS 65536   /* absorbed particles (per species) and ionisations per step and discharge */
#define EDUPIC_N_COUNTERS 19

/* counter indices for edupic_get_counters */
#define EDUPIC_C_ABS_E_POW 0    /* electrons absorbed at the powered electrode (x < 0) */
#define EDUPIC_C_ABS_E_GND 1    /* electrons absorbed at the grounded electrode (x > L) */
#define EDUPIC_C_ABS_I_POW 2
#define EDUPIC_C_ABS_I_GND 3
#define EDUPIC_C_COLL_E_ELA 4   /* e- + Ar elastic */
#define EDUPIC_C_COLL_E_EXC 5   /* e- + Ar excitation */
#define EDUPIC_C_COLL_E_ION 6   /* e- + Ar ionisation */
#define EDUPIC_C_COLL_I_ISO 7   /* Ar+ + Ar isotropic */
#define EDUPIC_C_COLL_I_BACK 8  /* Ar+ + Ar backward */
#define EDUPIC_C_SUBTHRESHOLD 9 /* inelastic picks below threshold, executed as elastic */
#define EDUPIC_C_CREATED 10     /* e-/Ar+ pairs created by ionisation */
#define EDUPIC_C_DROPPED 11     /* created pairs dropped at capacity */
#define EDUPIC_C_PUSH_E 12      /* electron pushes (particle-steps) */
#define EDUPIC_C_PUSH_I 13      /* ion pushes (particle-steps, ion steps only) */
#define EDUPIC_C_REFLECTED 14   /* electrons reflected elastically at an electrode (Sec. 5) */
#define EDUPIC_C_EMITTED_POW 15 /* secondary electrons emitted by ions at the powered electrode (Sec. 5) */
#define EDUPIC_C_EMITTED_GND 16 /* ... at the grounded electrode */
#define EDUPIC_C_NULL_TESTED 17 /* null-collision method: particles picked with probability P* */
#define EDUPIC_C_NULL_OVER 18   /* null-collision method: picked particles whose nu exceeded nu* */

/* ---------------------------------------------------------------- parameters */
/* One discharge (Table 1 / Table 2 quantities of the paper).  SI units except
 * the energy resolutions, which are in eV (Sec. 3.1). */
typedef struct {
    double gap_m;            /* electrode gap L */
    double pressure_pa;      /* gas pressure */
    double gas_temp_k;       /* gas temperature T_g */
    double area_m2;          /* electrode area A linking weight and density (1e-4 in the paper) */
    double weight;           /* superparticle weight W (>= 0) */
    int32_t n_grid;          /* grid points N_G, 3..EDUPIC_MAX_GRID */
    int32_t steps_per_cycle; /* N_T, a multiple of ion_subcycle */
    int32_t ion_subcycle;    /* N_SUB >= 1 */
    int32_t n_harmonics;     /* drive terms, 1..EDUPIC_MAX_HARMONICS */
    double cycle_freq_hz;    /* the RF cycle is one period of this frequency; dt_e = 1/(f N_T) */
    double harm_freq_hz[EDUPIC_MAX_HARMONICS]; /* V(t) = sum V_k cos(2 pi f_k t); each f_k an integer
                                                  multiple of cycle_freq_hz (0 = DC) */
    double harm_volt_v[EDUPIC_MAX_HARMONICS];
    uint64_t seed;           /* key of the counter-based random numbers */
    int32_t eepf_bins;       /* N_EEPF (2000 in the paper) */
    int32_t ifed_bins;       /* N_IFED (200) */
    double eepf_de_ev;       /* DE_EEPF (0.05 eV) */
    double ifed_de_ev;       /* DE_IFED (1 eV) */
    int64_t capacity_e;      /* particle capacity per species (MAX_N_P analogue, Sec. 3.1) */
    int64_t capacity_i;
    double e_exc_ev;         /* lumped excitation threshold (11.5 eV for Ar) */
    double e_ion_ev;         /* ionisation threshold (15.8 eV for Ar) */
    int32_t cs_entries;      /* capacity of the cross-section tables (CS_RANGES), shared by the object */
    /* Periodic cell sort (no counterpart in the paper; the particle loop's
     * memory locality): every sort_every ion subcycles (>= 0, 0 = off), after
     * the step whose index s becomes a multiple of sort_every * N_SUB, each
     * species is put in ascending order of its deposition cell floor(x/dx)
     * (Algorithm 2), keeping the slot order within a cell.  Slots, and with
     * them the random-number counters, follow the new order (the oracle
     * applies the same permutation).  Needs a scratch copy of the larger
     * species and one int per (2048-particle chunk, cell) in the arena. */
    int32_t sort_every;
    /* Surface processes (Sec. 5), index 0 = powered electrode (x = 0), 1 =
     * grounded (x = L); all zero switches them off (the reference discharge):
     *  - see_gamma[s]: probability that an Ar+ reaching electrode s emits an
     *    electron (0..1).  The electron starts at the electrode with a
     *    half-Maxwellian velocity of temperature see_te_ev pointing into the
     *    gap, and joins the electrons after the ionisation pairs of the step,
     *    in ascending order of the emitting ion's slot.
     *  - refl_eta[s]: probability that an electron reaching electrode s is
     *    reflected elastically (0..1): mirrored back into the gap (x -> -x,
     *    or 2L - x) with v_x reversed; absorbed if the mirror image is still
     *    outside the gap.
     * Random numbers: electron block 5 (reflection), ion blocks 5 (emission),
     * 6 and 7 (the emitted velocity). */
    double see_gamma[2];
    double refl_eta[2];
    double see_te_ev;        /* >= 0 */
    /* Null-collision method (Sec. 2.1.6; proposed in Sec. 5) instead of the
     * per-particle collision probability, per species: bit 0 (1) electrons,
     * bit 1 (2) ions, 3 both, 0 off (the paper's code).
     * nu* = the largest n sigma_tot v of the table, v taken at the top of
     * each energy bin (e-: lab speed; Ar+: relative speed, reduced mass);
     * P* = 1 - exp(-nu* dt).  A particle is picked when its collision-test
     * uniform u is below P*, and then collides when u / P* < nu / nu* (given
     * the pick, u / P* is uniform on [0, 1)); otherwise the collision is null.
     * An Ar+ draws its gas partner only when picked.  Energies past the table can exceed nu*; those particles always
     * collide when picked and are counted (EDUPIC_C_NULL_OVER). */
    int32_t null_collision;
    /* Spatio-temporal ("xt") diagnostics (Sec. 3.5): N_XT time bins per RF
     * cycle (N_T a multiple of it, N_BIN = N_T / N_XT steps per bin), 0 = off.
     * Read with edupic_get_xt. */
    int32_t xt_bins;
} edupic_params;

typedef struct edupic_sim edupic_sim;

/* ---------------------------------------------------------------- lifecycle */

/* Bytes of device memory a simulation of n discharges needs (Sec. 3.1
 * static arrays, here sized from capacities).  params: host array of n
 * parameter sets.  precision: EDUPIC_FP64 or EDUPIC_FP32.  Writes *bytes. */
int edupic_arena_bytes(int n_discharges, const edupic_params *params, int precision, size_t *bytes);

/* Create a simulation of n discharges that are stepped together by one set of
 * kernel launches per time step.  device_arena: caller-owned device memory of
 * at least edupic_arena_bytes bytes, 256-byte aligned; it must stay allocated
 * until edupic_destroy.  cuda_stream: a cudaStream_t (NULL = legacy default
 * stream).  All discharges must share ion_subcycle and cs_entries.  The
 * particle arrays start empty; the cross sections must be set before the
 * first step.  On success *out owns host-side state only. */
int edupic_create(int n_discharges, const edupic_params *params, int precision, void *device_arena,
                  size_t arena_bytes, void *cuda_stream, edupic_sim **out);

/* Release the host-side state (and CUDA graphs).  The arena is not freed. */
int edupic_destroy(edupic_sim *sim);

/* Cross sections (Sec. 3.2), shared by every discharge of the object.
 * species: EDUPIC_ELECTRONS (n_proc 3: elastic, excitation, ionisation, by
 * LAB energy) or EDUPIC_IONS (n_proc 2: isotropic, backward, by COM energy).
 * sigma_m2: host, [n_proc][n_entries] row-major, in m^2, at energies k*de_ev.
 * n_entries <= cs_entries.  Energies beyond the table use the last entry. */
int edupic_set_cross_sections(edupic_sim *sim, int species, int n_proc, int n_entries, double de_ev,
                              const double *sigma_m2);

/* The electrons' collision-test bound that edupic_set_cross_sections forms
 * (host computation only, no device; for inspection).  The direct test of
 * Algorithm 6 compares the test uniform with P_coll = 1 - exp(-n sigma_tot v
 * dt); the particle kernel first compares it with a bound per v^2 bucket:
 * the bucket of a squared speed w is the exponent and top five mantissa bits
 * of w in the particle precision (FP32: bits >> 18; FP64: bits >> 47),
 * clamped to [*base_out, *base_out + *n_out - 1].  Entry j - *base_out of
 * table_out holds the largest sigma_tot,k times the speed at the bucket's
 * top over every entry k a w of the bucket can index (nearest entry, one
 * entry of margin each side), widened by 1e-6 and rounded up in the
 * particle precision; the kernel multiplies it by n dt.  The last bucket is
 * +inf.  sigma_sum: host, n_entries values of the summed electron cross
 * sections (m^2) at energies k*de_ev; table_out: host, EDUPIC_BOUND_BUCKETS
 * doubles (entries past *n_out are +inf).  EDUPIC_EINVAL on a bad argument. */
#define EDUPIC_BOUND_BUCKETS 2048
int edupic_electron_bound_table(int precision, int n_entries, double de_ev, const double *sigma_sum,
                                double *table_out, int *base_out, int *n_out);

/* Replace the particles of one species of discharge d (host FP64 arrays of n
 * entries; stored as FP32 in EDUPIC_FP32 mode).  The densities of that species
 * and the field of the current step are recomputed (Algorithms 2-3), as the
 * paper does after seeding or loading particles (Algorithm 1). */
int edupic_load_particles(edupic_sim *sim, int d, int species, int64_t n, const double *x, const double *vx,
                          const double *vy, const double *vz);

/* init(N_INIT) of Algorithm 1: replace both species of discharge d by n_init
 * electrons and n_init Ar+ ions at random positions in the gap with zero
 * velocities, and form the densities and the field of the current step.
 * Positions: x = L R01, R01 from block 9 of each particle's counter-based
 * random numbers (slot, current step, species), so the state depends only on
 * the seed and the step.  EDUPIC_ECAPACITY beyond either capacity.
 * Synchronises the stream. */
int edupic_seed(edupic_sim *sim, int d, int64_t n_init);

/* ---------------------------------------------------------------- stepping */

/* Enqueue n_steps PIC/MCC time steps (Sec. 2.1, Fig. 2) of every discharge.
 * Ions are pushed and collide on steps whose index within the RF cycle is a
 * multiple of N_SUB (ion subcycling).  measure != 0 accumulates the
 * diagnostics of Sec. 3.5 (time-averaged densities and potential, EEPF in the
 * central 10% of the gap, IFEDF at both electrodes). */
int edupic_step(edupic_sim *sim, int64_t n_steps, int measure);

/* Enqueue n_cycles RF cycles (n_cycles * N_T steps), as do_one_cycle() is
 * repeated by the paper's main() (Algorithm 1).  Requires all discharges to
 * share steps_per_cycle. */
int edupic_run_cycles(edupic_sim *sim, int n_cycles, int measure);

/* Wait for the stream and return the first device-side error (or OK). */
int edupic_synchronize(edupic_sim *sim);

/* Self-test of the bounded waits (no counterpart in the paper: every wait of
 * the particle kernel on its asynchronous copies gives up after a limit and
 * records an error instead of waiting forever).  One block waits, with the
 * same bounded wait, limit_ns nanoseconds (1e3..1e9) on a barrier that
 * nothing ever arrives on, records the expiry in discharge d's error bits
 * and returns.  Returns EDUPIC_ETIMEOUT (as edupic_synchronize will from then
 * on: the error bits are sticky).  The GPU context stays usable. */
int edupic_selftest_wait_expiry(edupic_sim *sim, int d, int64_t limit_ns);

/* Run n_steps exactly as edupic_step does, but launch by launch (no graph)
 * with a CUDA event pair on the object's stream around every kernel, and
 * synchronise after each step.  out_ms[0..2] receive the summed device time
 * (ms) of the electron particle kernel, the ion particle kernel and the
 * per-discharge finalize kernel (compaction, append, field solve);
 * launches[0..2] their launch counts.  Both arrays are host memory. */
int edupic_profile_steps(edupic_sim *sim, int64_t n_steps, int measure, double out_ms[3], int64_t launches[3]);

/* Use (1, default) or bypass (0) the CUDA graph that replays one ion
 * subcycle of kernel launches.  Results are identical either way. */
int edupic_set_graphs(edupic_sim *sim, int enable);
/* Writes 1 if graph replay is in use (as set, or as edupic_autotune chose). */
int edupic_get_graphs(edupic_sim *sim, int *enabled);

/* Launch of the particle kernels (no counterpart in the paper, whose
 * particle loops are serial).  The particle kernel runs a persistent grid
 * of thread blocks that share the particle tiles of all discharges: the
 * resident limit (blocks per SM that fit the registers and shared memory,
 * times the SM count) of its launch shape.  edupic_set_push_grid accepts
 * blocks = 0 or that limit (anything else is EDUPIC_EINVAL: smaller
 * persistent grids stalled on large batches and are not offered).
 * edupic_get_push_grid writes the grids of the electron and ion kernels to
 * out[0..1] (host memory). */
int edupic_set_push_grid(edupic_sim *sim, int species, int blocks);
int edupic_get_push_grid(edupic_sim *sim, int out[2]);

/* Launch shapes of the particle kernel: EDUPIC_PUSH_SHAPES compiled
 * variants that differ in threads per block, tile-ring stages and the
 * blocks per SM their register budget targets; every shape gives the same
 * particles, densities, counters and histograms.  edupic_set_push_shape
 * selects shape 0..EDUPIC_PUSH_SHAPES-1 for one species (EDUPIC_EINVAL if
 * out of range or if it does not fit the object's grid size and tables);
 * edupic_get_push_shape writes the shapes in use (out[0..1], host memory);
 * edupic_describe_push_shape writes a shape's threads per block, ring
 * stages and targeted blocks per SM (pointers may be NULL). */
#define EDUPIC_PUSH_SHAPES 4
int edupic_set_push_shape(edupic_sim *sim, int species, int shape);
int edupic_get_push_shape(edupic_sim *sim, int out[2]);
int edupic_describe_push_shape(int precision, int shape, int *threads, int *stages, int *min_blocks);

/* Autotuner of the launch (block and tile sizes picked by timing).  First,
 * every launch shape that fits is run for `subcycles` ion subcycles launch
 * by launch with an event pair around each particle-kernel launch, and each
 * species keeps the shape of its fastest mean launch.  Then it times
 * `subcycles` ion subcycles replayed through one CUDA graph per ion
 * subcycle against the same launched kernel by kernel, and keeps the faster
 * stepping mode.  Results are identical for every choice.  The trial steps
 * are real simulation steps (the simulation advances by
 * (fitting shapes + 2) x (subcycles + 1) ion subcycles, measured if
 * `measure`); call it at the start of a run, at ion phase 0 (else
 * EDUPIC_ESTATE).  out_blocks[0..1] and out_ms_per_step (host, may be NULL)
 * receive the grids in use and the trial time per step of the faster
 * mode. */
int edupic_autotune(edupic_sim *sim, int subcycles, int measure, int out_blocks[2], double *out_ms_per_step);

/* ---------------------------------------------------------------- read-back (synchronising) */

/* Live particle counts and the global step index of discharge d. */
int edupic_get_counts(edupic_sim *sim, int d, int64_t *n_e, int64_t *n_i, int64_t *step);

/* Copy up to cap particles of one species into host arrays (FP64).  Writes
 * *n_out with the live count; slots follow the canonical compaction order. */
int edupic_get_particles(edupic_sim *sim, int d, int species, int64_t cap, double *x, double *vx, double *vy,
                         double *vz, int64_t *n_out);

/* Fields that the next step uses (Algorithms 2-3): densities n_e, n_i
 * (m^-3), potential phi (V), field E (V/m), and the fixed-point deposition
 * sums q_e, q_i (2^32 units per particle).  Any pointer may be NULL; each
 * non-NULL array holds n_grid entries. */
int edupic_get_fields(edupic_sim *sim, int d, double *n_e, double *n_i, double *phi, double *efield, int64_t *q_e,
                      int64_t *q_i);

/* Time-averaged densities and potential over the measured steps, and the raw
 * EEPF / IFEDF histograms (Sec. 3.5).  Any pointer may be NULL. */
int edupic_get_diagnostics(edupic_sim *sim, int d, double *ne_avg, double *ni_avg, double *phi_avg,
                           int64_t *eepf_counts, int64_t *ifed_pow_counts, int64_t *ifed_gnd_counts,
                           int64_t *measured_steps);

/* Normalised EEPF f(eps) (sum f sqrt(eps) dE = 1) and IFEDFs F(eps)
 * (sum F dE = 1) at bin centres (Sec. 3.5).  Any output may be NULL. */
int edupic_get_eepf(edupic_sim *sim, int d, double *energy_ev, double *f);
int edupic_get_ifed(edupic_sim *sim, int d, double *energy_ev, double *f_pow, double *f_gnd);

/* Event counters (EDUPIC_C_* indices), accumulated since creation. */
int edupic_get_counters(edupic_sim *sim, int d, int64_t out[EDUPIC_N_COUNTERS]);

/* Clear the measured diagnostics of discharge d. */
int edupic_reset_diagnostics(edupic_sim *sim, int d);

/* Power absorption of Sec. 3.5: the space and time average of j E for
 * electrons (out[0]) and Ar+ (out[1]) over the gap and the measured steps,
 * in W/m^3, from the field's work on every measured push, q E_x v_c dt with
 * v_c = (v_old + v_new) / 2 (E_x gathered at the position before the push):
 * W / (A L T_meas) times that sum, T_meas = measured steps x dt_e.  out is
 * host memory; zero before any measured step.  The sums are added in an
 * order that depends on the launch, so results agree to rounding, not bit
 * for bit, between runs. */
int edupic_get_power(edupic_sim *sim, int d, double out[2]);

/* DC self-bias (Sec. 5: the bias is adjusted in an iteration until the
 * currents of the oppositely charged particles reaching an electrode
 * compensate on time average).  The bias is a constant voltage added to the
 * drive at the powered electrode: phi_0 = V(t) + v_bias.
 *
 * edupic_set_bias sets it for discharge d (finite volts; 0 at creation) and
 * forms the field of the coming step again with it.  edupic_get_bias reads it.
 *
 * edupic_self_bias_step is one iteration for every discharge: it runs n_steps
 * time steps (edupic_step, measuring if `measure`), counts over them the ions
 * N_i and electrons N_e absorbed at the powered electrode and the secondary
 * electrons N_s it emitted, and for each discharge d with gain_v[d] != 0 sets
 *     v_bias += gain_v[d] * (N_i - N_e + N_s) / (N_i + N_e + N_s)
 * (the normalised net positive charge the electrode received; unchanged when
 * nothing arrived).  gain_v: host, nd values (volts; 0 = leave d alone).
 * v_bias: host, nd values written with the new biases, or NULL.  Take n_steps
 * a multiple of the RF cycles so that the window is a time average; the
 * iteration converges for gains small against the bias scale (a few volts
 * for the discharges here).  Synchronises the stream; device errors are
 * returned. */
int edupic_set_bias(edupic_sim *sim, int d, double v_bias);
int edupic_get_bias(edupic_sim *sim, int d, double *v_bias);
int edupic_self_bias_step(edupic_sim *sim, int64_t n_steps, int measure, const double *gain_v, double *v_bias);

/* Spatio-temporal ("xt") diagnostics of Sec. 3.5, for a discharge created
 * with xt_bins = N_XT > 0.  Every measured step adds to time bin
 * b = (t mod N_T) / N_BIN: the grid quantities after the field solve, and in
 * the particle push the particle quantities at the position x(t) with the
 * time-centred velocity v_c = (v(t-1/2) + v(t+1/2)) / 2, weighted to the two
 * grid points like the density deposition (Sec. 2.1.1); ionisations add at
 * the collision position.  Maps are averages over the measured steps of each
 * bin (ions: over the ion steps).  quantity:
 *   EDUPIC_XT_POT, EDUPIC_XT_EFIELD  potential (V), electric field (V/m)
 *   EDUPIC_XT_NE, EDUPIC_XT_NI       densities (m^-3)
 *   EDUPIC_XT_JE, EDUPIC_XT_JI       current densities q n <v_c,x> (A/m^2)
 *   EDUPIC_XT_POWERE, _POWERI        power absorption j E (W/m^3), the product
 *                                    of the current and field maps
 *   EDUPIC_XT_MEANEE, _MEANEI        mean energies (1/2) m <|v_c|^2> (eV; 0
 *                                    where no particle was counted)
 *   EDUPIC_XT_IONIZ                  ionisation rate (m^-3 s^-1)
 * out: host, n_grid x xt_bins doubles, row-major (row = grid point, column =
 * time bin).  Bins that no measured step reached are 0.  EDUPIC_ESTATE if
 * the discharge has no xt diagnostics.  Synchronises the stream.
 * (The request server does not keep xt maps: requests with xt_bins > 0 are
 * refused there.) */
#define EDUPIC_XT_POT 0
#define EDUPIC_XT_EFIELD 1
#define EDUPIC_XT_NE 2
#define EDUPIC_XT_NI 3
#define EDUPIC_XT_JE 4
#define EDUPIC_XT_JI 5
#define EDUPIC_XT_POWERE 6
#define EDUPIC_XT_POWERI 7
#define EDUPIC_XT_MEANEE 8
#define EDUPIC_XT_MEANEI 9
#define EDUPIC_XT_IONIZ 10
#define EDUPIC_XT_QUANTITIES 11
int edupic_get_xt(edupic_sim *sim, int d, int quantity, double *out);

/* Accuracy and stability conditions of Sec. 2.2 (the checks the paper's
 * code writes to info.txt, Sec. 3.5), evaluated for discharge d from its
 * measured diagnostics (so after measured steps, else EDUPIC_ESTATE):
 *  1. dx / lambda_D <= 1, lambda_D from the peak time-averaged n_e and the
 *     effective temperature kT_e = 2/3 of the mean EEPF energy;
 *  2. omega_pe dt_e < 2 at the peak time-averaged n_e;
 *  3. the largest collision probability per step, 1 - exp(-n_gas
 *     max(sigma_tot v) dt), below 0.05 for e- (dt_e) and Ar+ (dt_i), the
 *     maximum taken over the tables (v: e- speed of the entry's energy,
 *     Ar+ relative speed with the reduced mass);
 *  4. the energies at which v dt = dx (e-: dt_e, Ar+: dt_i): the CFL limit,
 *     to be compared by the user with where the EEPF has decayed.
 * Writes *out (host) and returns EDUPIC_OK, or EDUPIC_ESTABILITY if one of
 * 1-3 fails (out->failed: bit 0, 1, 2).  Opt-in: nothing else calls it. */
typedef struct {
    double debye_ratio;   /* dx / lambda_D */
    double wpe_dt;        /* omega_pe dt_e */
    double pcoll_max_e;   /* largest e- collision probability per electron step */
    double pcoll_max_i;   /* largest Ar+ collision probability per ion step */
    double cfl_max_ev_e;  /* e- energy (eV) with v dt_e = dx */
    double cfl_max_ev_i;  /* Ar+ energy (eV) with v dt_i = dx */
    double te_ev;         /* effective electron temperature used (eV) */
    double ne_max;        /* peak time-averaged electron density used (m^-3) */
    int failed;           /* bit 0: condition 1, bit 1: condition 2, bit 2: condition 3 */
    int reserved;
} edupic_accuracy;

int edupic_check_accuracy(edupic_sim *sim, int d, edupic_accuracy *out);

/* ---------------------------------------------------------------- checkpoint */

/* Save / restore the state of discharge d (counts, step index, particle
 * coordinates), the analogue of picdata.bin (Algorithm 1).  The file has a
 * versioned header; a restore recomputes the densities and field.
 * edupic_load_state reads and checks the whole file before it changes
 * anything: EDUPIC_EIO for a file that is missing, short, longer than its
 * counts, of another version or another N_G; EDUPIC_ECAPACITY for counts
 * above the capacity; EDUPIC_ESTATE for a step of another ion-subcycle
 * phase than the object's; EDUPIC_EINVAL for a position outside [0, L] or a
 * non-finite velocity.  On any error the simulation is unchanged. */
int edupic_save_state(edupic_sim *sim, int d, const char *path);
int edupic_load_state(edupic_sim *sim, int d, const char *path);

/* ---------------------------------------------------------------- request server */

/* Continuous batching of independent discharge simulations on one GPU.
 * (The paper runs one simulation per process and has no counterpart: its
 * program flow of init, N RF cycles and read-out, Sec. 3.5 and Algorithm 1,
 * is what each request asks for.)
 *
 * A server keeps up to max_slots requests resident.  Each request is a full
 * simulation (edupic_params, initial particles, n_cycles RF cycles with the
 * diagnostics of Sec. 3.5 accumulated over the whole run).  The particle
 * and grid memory of a request is carved from the caller's arena when it is
 * admitted and returned when it finishes, so the arena size is the HBM
 * budget.  All running requests advance together, one push launch per
 * species and one finalize launch per time step, and each stops at its own
 * target step: a request's results are the same whatever else runs beside
 * it.  Requests are admitted in submission order at ion-subcycle boundaries
 * while a slot and enough arena memory are free. */
typedef struct edupic_server edupic_server;

typedef struct {
    int max_slots;     /* requests resident at once, 1..EDUPIC_MAX_DISCHARGES */
    int max_grid;      /* largest N_G a request may use, 3..EDUPIC_MAX_GRID */
    int max_eepf_bins; /* largest EEPF bin count, 1..EDUPIC_MAX_EEPF_BINS */
    int ion_subcycle;  /* N_SUB shared by every request */
    int cs_entries;    /* cross-section table length shared by every request */
    int reserved;
} edupic_server_config;

#define EDUPIC_REQ_QUEUED 0
#define EDUPIC_REQ_RUNNING 1
#define EDUPIC_REQ_DONE 2
#define EDUPIC_REQ_FAILED 3

typedef struct {
    int state;            /* EDUPIC_REQ_* */
    int status;           /* EDUPIC_OK, or the error that ended the request */
    int slot;             /* slot it runs / ran in, -1 while queued */
    int reserved;
    int64_t steps_target; /* n_cycles * N_T */
    int64_t steps_done;   /* time steps run (final value once done) */
    int64_t n_e, n_i;     /* particle counts: initial while queued/running, final once done */
    int64_t bytes;        /* arena bytes the request holds while running */
    double t_submit, t_admit, t_done; /* seconds on the server's monotonic clock, -1 if not yet */
} edupic_request_info;

typedef struct {
    double now;           /* seconds since the server was created */
    int64_t steps_run;    /* time steps enqueued since creation */
    int64_t heap_bytes, heap_used;
    int running, queued;
} edupic_server_stats_t;

/* Arena bytes for a server with `heap_bytes` of request memory. */
int edupic_server_arena_bytes(const edupic_server_config *cfg, int precision, size_t heap_bytes, size_t *bytes);

/* Create a server in a caller-owned device arena (256-byte aligned; the
 * caller keeps it alive until edupic_server_destroy).  The part of the arena
 * beyond the fixed shared region is the request heap.  Work runs on
 * cuda_stream (a non-default stream: steps are replayed as CUDA graphs).
 * EDUPIC_ENOMEM if the arena cannot hold the shared region. */
int edupic_server_create(const edupic_server_config *cfg, int precision, void *device_arena, size_t arena_bytes,
                         void *cuda_stream, edupic_server **out);
int edupic_server_destroy(edupic_server *srv);

/* Cross sections shared by all requests (as edupic_set_cross_sections);
 * EDUPIC_ESTATE while a request is running. */
int edupic_server_set_cross_sections(edupic_server *srv, int species, int n_proc, int n_entries, double de_ev,
                                     const double *sigma_m2);

/* Arena bytes a request with these parameters holds while it runs. */
int edupic_server_request_bytes(const edupic_server *srv, const edupic_params *p, size_t *bytes);

/* Queue a request: parameters p (checked as edupic_create does, plus
 * n_grid <= max_grid, eepf_bins <= max_eepf_bins and the server's N_SUB and
 * table length), n_cycles >= 1 RF cycles, and the initial particles:
 * e[0..3] = x, vx, vy, vz of n_e electrons and i[0..3] of n_i ions, host
 * FP64 arrays copied during the call (positions in [0, L]).  Returns a
 * ticket.  EDUPIC_ENOMEM if the request can never fit the arena,
 * EDUPIC_ECAPACITY if a count exceeds its capacity. */
int edupic_server_submit(edupic_server *srv, const edupic_params *p, int n_cycles, int64_t n_e,
                         const double *const e[4], int64_t n_i, const double *const i[4], uint64_t *ticket);

/* One scheduling round: wait for the steps enqueued by the previous call,
 * retire requests that reached their target step (their results are read
 * back to host memory and their arena memory freed), admit queued requests,
 * then enqueue n_subcycles ion subcycles (n_subcycles * N_SUB time steps)
 * for every running request and return without waiting for them.  Writes
 * the running and queued counts after admission. */
int edupic_server_advance(edupic_server *srv, int n_subcycles, int *n_running, int *n_queued);

/* State, counts and timestamps of a request. */
int edupic_server_info(edupic_server *srv, uint64_t ticket, edupic_request_info *info);

/* Results of a finished request, as edupic_get_diagnostics and
 * edupic_get_counters give them: time-averaged n_e, n_i, phi (n_grid each),
 * EEPF counts (eepf_bins), IFED counts per electrode (ifed_bins each),
 * counters and the number of measured steps.  Any pointer may be NULL.
 * EDUPIC_ESTATE while the request is queued or running; the request's error
 * if it failed. */
int edupic_server_result(edupic_server *srv, uint64_t ticket, double *ne_avg, double *ni_avg, double *phi_avg,
                         int64_t *eepf_counts, int64_t *ifed_pow_counts, int64_t *ifed_gnd_counts,
                         int64_t counters[EDUPIC_N_COUNTERS], int64_t *measured_steps);

/* Forget a request.  A queued request leaves the queue.  A running request
 * is cancelled: the call waits for the steps already enqueued on the
 * server's stream, then returns the request's slot and heap memory; the
 * other running requests are not affected (their results stay the same).  A
 * finished or failed request loses its host-side results.  EDUPIC_EINVAL for
 * an unknown ticket. */
int edupic_server_release(edupic_server *srv, uint64_t ticket);

/* Clock, step count, heap use and slot occupancy. */
int edupic_server_stats(edupic_server *srv, edupic_server_stats_t *out);

/* ---------------------------------------------------------------- no-allocation entry point */

/* Densities, potential and field of given particle positions, computed
 * without allocating any device memory.  (The paper has no counterpart: it
 * is an interface for callers that cannot call cudaMalloc mid-run, e.g.
 * code whose device memory is pre-budgeted by another framework's pool,
 * where an allocation would fail or break the budget, or code inside a
 * plugin or a real-time loop that must not touch the allocator, which can
 * block on the device.)
 *
 * Computes what edupic_load_particles followed by edupic_get_fields gives in
 * EDUPIC_FP64 mode: fixed-point deposition of x_e and x_i (Algorithm 2) and
 * the Poisson solve with phi_0 = V(t) at within-cycle step step % N_T
 * (Algorithm 3).  Uses p->gap_m, area_m2, weight, n_grid, steps_per_cycle,
 * cycle_freq_hz and the harmonics.
 *
 * x_e, x_i: device FP64 positions in [0, L] (n_e, n_i entries, may be NULL
 * when the count is 0).  A position outside [0, L], or not a number, is
 * reported as EDUPIC_EINVAL; the outputs are then unspecified.
 * n_e_out, n_i_out (m^-3), phi_out (V), efield_out (V/m): device FP64 arrays
 * of n_grid entries, written by the call.
 * cuda_stream: cudaStream_t (NULL = legacy default stream); the call
 * synchronises it before returning (it reads the position check back).
 *
 * Working memory is one fixed array of 49,408 bytes in the library's device
 * image, held by every GPU that loads the library until the process exits;
 * n_grid above EDUPIC_MAX_GRID (2048) is rejected with EDUPIC_ETOOBIG.  The
 * first call on a device looks up that array's device address (a CUDA
 * runtime query), so make the first call before any stream capture.  The
 * array is shared by all calls and keeps the last call's contents (each call
 * zeroes what it accumulates into first); calls that overlap on the GPU race
 * on it, so issue them one at a time per device.  No cudaMalloc, cudaFree or
 * allocating library routine is called. */
int edupic_fields_noalloc(const edupic_params *p, int64_t step, const double *x_e, int64_t n_e, const double *x_i,
                          int64_t n_i, double *n_e_out, double *n_i_out, double *phi_out, double *efield_out,
                          void *cuda_stream);

/* Text for a status code. */
const char *edupic_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* EDUPIC_H */
