// Host side of the C ABI declared in include/edupic.h: parameter checks,
// arena layout, descriptor upload, step scheduling (with one CUDA graph per
// ion subcycle), read-back and checkpoints.  No particle arithmetic runs here.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "edupic_host.h"

using namespace edupic;
using namespace edupic::host;

namespace edupic {
namespace host {

constexpr double kQE = 1.602176634e-19;
constexpr double kME = 9.1093837015e-31;
constexpr double kEPS0 = 8.8541878128e-12;
constexpr double kKB = 1.380649e-23;
constexpr double kAMU = 1.66053906660e-27;
constexpr double kArMassU = 39.948;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

long long padded(long long cap) { return (cap + kTileAlign - 1) / kTileAlign * kTileAlign; }


Layout layout_of(const edupic_params &p, size_t elem)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t n) {
        const size_t at = o;
        o = align_up(o + n, kAlign);
        return at;
    };
    const long long cap[2] = {padded(p.capacity_e), padded(p.capacity_i)};
    for (int s = 0; s < 2; ++s) {
        L.x[s] = take(cap[s] * elem);
        L.vx[s] = take(cap[s] * elem);
        L.vy[s] = take(cap[s] * elem);
        L.vz[s] = take(cap[s] * elem);
    }
    const size_t ng = (size_t)p.n_grid;
    L.q_e = take(ng * 8);
    L.q_i = take(ng * 8);
    L.acc_e = take(ng * 8);
    L.acc_i = take(ng * 8);
    L.n_e = take(ng * 8);
    L.n_i = take(ng * 8);
    L.phi = take(ng * 8);
    L.ef = take(ng * 8);
    L.ef_t = take(ng * elem);
    L.f_cur = take(ng * 8);
    L.fs = take(sizeof(FieldState));
    L.sum_qe = take(ng * 8);
    L.sum_qi = take(ng * 8);
    L.sum_f = take(ng * 8);
    L.avg = take(3 * ng * 8);
    L.eepf = take((size_t)kEepfStripes * p.eepf_bins * 8);
    L.ifed_pow = take((size_t)p.ifed_bins * 8);
    L.ifed_gnd = take((size_t)p.ifed_bins * 8);
    L.power = take(2 * sizeof(double));
    L.holes[0] = take((size_t)kEvents * 4);
    L.holes[1] = take((size_t)kEvents * 4);
    L.prod_parent = take((size_t)kEvents * 4);
    L.sort_buf = take((size_t)kEvents * 4);
    L.prod_x = take((size_t)kEvents * elem);
    for (int c = 0; c < 3; ++c) L.prod_ve[c] = take((size_t)kEvents * elem);
    for (int c = 0; c < 3; ++c) L.prod_vi[c] = take((size_t)kEvents * elem);
    L.vdrive = take((size_t)p.steps_per_cycle * 8);
    if (p.xt_bins > 0) {
        const size_t m = ng * (size_t)p.xt_bins;
        L.xt_bytes = 9 * m * 8 + 4 * (size_t)p.xt_bins * 8;
        L.xt = take(L.xt_bytes);
    }
    if (p.sort_every > 0) {
        const long long cmax = std::max(cap[0], cap[1]);
        L.sort_cnt = take((size_t)((cmax + kSortChunk - 1) / kSortChunk) * ng * 4);
        for (int c = 0; c < 4; ++c) L.sort_tmp[c] = take((size_t)cmax * elem);
    }
    L.emit = p.see_gamma[0] > 0.0 || p.see_gamma[1] > 0.0;
    if (L.emit) {
        L.emit_parent = take((size_t)kEvents * 4);
        L.emit_x = take((size_t)kEvents * elem);
        for (int c = 0; c < 3; ++c) L.emit_v[c] = take((size_t)kEvents * elem);
    }
    L.bytes = o;
    return L;
}

bool is_multiple(double f, double base)
{
    if (f == 0.0) return true;
    const double r = f / base;
    return r >= 0.5 && std::fabs(r - std::nearbyint(r)) <= 1e-9 * r;
}

int check_params(int nd, const edupic_params *ps, int precision)
{
    if (nd < 1 || nd > EDUPIC_MAX_DISCHARGES || !ps) return EDUPIC_EINVAL;
    if (precision != EDUPIC_FP64 && precision != EDUPIC_FP32) return EDUPIC_EINVAL;
    for (int d = 0; d < nd; ++d) {
        const edupic_params &p = ps[d];
        if (!(p.gap_m > 0) || !(p.pressure_pa >= 0) || !(p.gas_temp_k > 0) || !(p.area_m2 > 0) || !(p.weight >= 0))
            return EDUPIC_EINVAL;
        if (p.n_grid < 3 || p.n_grid > EDUPIC_MAX_GRID) return EDUPIC_EINVAL;
        if (p.steps_per_cycle < 1 || p.ion_subcycle < 1 || p.steps_per_cycle % p.ion_subcycle) return EDUPIC_EINVAL;
        if (p.ion_subcycle != ps[0].ion_subcycle || p.cs_entries != ps[0].cs_entries) return EDUPIC_EINVAL;
        if (p.n_harmonics < 0 || p.n_harmonics > EDUPIC_MAX_HARMONICS || !(p.cycle_freq_hz > 0)) return EDUPIC_EINVAL;
        for (int k = 0; k < p.n_harmonics; ++k)
            if (!(p.harm_freq_hz[k] >= 0) || !is_multiple(p.harm_freq_hz[k], p.cycle_freq_hz)) return EDUPIC_EINVAL;
        if (p.eepf_bins < 1 || p.eepf_bins > EDUPIC_MAX_EEPF_BINS || !(p.eepf_de_ev > 0)) return EDUPIC_EINVAL;
        if (p.ifed_bins < 1 || p.ifed_bins > EDUPIC_MAX_IFED_BINS || !(p.ifed_de_ev > 0)) return EDUPIC_EINVAL;
        if (p.capacity_e < 1 || p.capacity_i < 1 || p.capacity_e > (1ll << 31) - 2 * kTileAlign ||
            p.capacity_i > (1ll << 31) - 2 * kTileAlign)
            return EDUPIC_EINVAL;
        if (p.cs_entries < 1 || p.cs_entries > EDUPIC_MAX_CS_ENTRIES) return EDUPIC_EINVAL;
        if (!(p.e_exc_ev >= 0) || !(p.e_ion_ev > 0)) return EDUPIC_EINVAL;
        for (int s = 0; s < 2; ++s)
            if (!(p.see_gamma[s] >= 0 && p.see_gamma[s] <= 1) || !(p.refl_eta[s] >= 0 && p.refl_eta[s] <= 1))
                return EDUPIC_EINVAL;
        if (!(p.see_te_ev >= 0) || !(p.see_te_ev < 1e6)) return EDUPIC_EINVAL;
        if (p.null_collision < 0 || p.null_collision > 3) return EDUPIC_EINVAL;
        if (p.sort_every < 0) return EDUPIC_EINVAL;
        if (p.xt_bins < 0 || (p.xt_bins > 0 && p.steps_per_cycle % p.xt_bins != 0) ||
            (int64_t)p.xt_bins * p.n_grid > (1 << 24))
            return EDUPIC_EINVAL;
    }
    return EDUPIC_OK;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? EDUPIC_OK : EDUPIC_ECUDA; }

}  // namespace host
}  // namespace edupic


namespace edupic {
namespace host {

size_t shared_bytes(int nd, size_t elem, int cs_entries)
{
    size_t o = align_up(sizeof(DischargeDev) * nd, kAlign);
    o += align_up(sizeof(Ctrl) * nd, kAlign);                  // packed counts and counters
    o += 2 * align_up((size_t)cs_entries * elem, kAlign);      // sigsum
    o += 2 * align_up((size_t)cs_entries * 2 * elem, kAlign);  // thr1, thr2
    o += 2 * align_up((size_t)kCoarse * elem, kAlign);         // coarse maxima
    o += 2 * align_up((size_t)kCoarse * elem, kAlign);         // prefix maxima of sigma_tot * v
    return o;
}

void fill_desc(edupic_sim *S, int d)
{
    const edupic_params &p = S->params[d];
    const Layout &L = S->layouts[d];
    unsigned char *b = S->arena + S->base[d];
    DischargeDev D{};
    // Section 3.1 / Table 1 derived quantities, in the paper's expression order.
    const double ar_mass = kArMassU * kAMU;
    D.L = p.gap_m;
    D.dx = p.gap_m / (p.n_grid - 1);
    D.inv_dx = 1.0 / D.dx;
    D.dt_e = 1.0 / (p.cycle_freq_hz * p.steps_per_cycle);
    D.dt_i = p.ion_subcycle * D.dt_e;
    D.factor_w = p.weight / (p.area_m2 * D.dx);
    D.factor_e = D.dt_e / kME * kQE;
    D.factor_i = D.dt_i / ar_mass * kQE;
    D.n_gas = p.pressure_pa / (kKB * p.gas_temp_k);
    D.sig_th = std::sqrt(kKB * p.gas_temp_k / ar_mass);
    D.ar_mass = ar_mass;
    D.mu_e = kME * ar_mass / (kME + ar_mass);
    const double mu_arar = ar_mass / 2.0;
    D.half_me = 0.5 * kME;
    D.half_mar = 0.5 * ar_mass;
    D.half_mu_e = 0.5 * D.mu_e;
    D.half_mu_arar = 0.5 * mu_arar;
    D.e_exc = p.e_exc_ev;
    D.e_ion = p.e_ion_ev;
    D.eepf_lo = 0.45 * p.gap_m;
    D.eepf_hi = 0.55 * p.gap_m;
    D.eepf_de = p.eepf_de_ev;
    D.ifed_de = p.ifed_de_ev;
    D.cs_de_e = S->desc.size() > (size_t)d ? S->desc[d].cs_de_e : 1.0;
    D.cs_de_i = S->desc.size() > (size_t)d ? S->desc[d].cs_de_i : 1.0;
    D.poisson_c = D.dx * D.dx * kQE * D.factor_w / (kEPS0 * 4294967296.0);
    D.rho_c = kQE * D.factor_w / 4294967296.0;
    for (int k = 0; k < EDUPIC_MAX_HARMONICS; ++k) {
        D.harm_freq[k] = k < p.n_harmonics ? p.harm_freq_hz[k] : 0.0;
        D.harm_volt[k] = k < p.n_harmonics ? p.harm_volt_v[k] : 0.0;
    }
    D.Lf = (float)D.L;
    D.inv_dxf = (float)D.inv_dx;
    D.dt_ef = (float)D.dt_e;
    D.dt_if = (float)D.dt_i;
    D.factor_ef = (float)D.factor_e;
    D.factor_if = (float)D.factor_i;
    D.n_gasf = (float)D.n_gas;
    D.sig_thf = (float)D.sig_th;
    D.e_of_v2_ef = (float)(0.5 * kME / kQE);
    D.e_of_v2_if = (float)(0.5 * ar_mass / kQE);
    D.e_of_g2_if = (float)(0.5 * mu_arar / kQE);
    D.mu_ef = (float)D.mu_e;
    D.e_excf = (float)p.e_exc_ev;
    D.e_ionf = (float)p.e_ion_ev;
    D.eepf_lof = (float)D.eepf_lo;
    D.eepf_hif = (float)D.eepf_hi;
    D.inv_eepf_def = (float)(1.0 / p.eepf_de_ev);
    D.inv_ifed_def = (float)(1.0 / p.ifed_de_ev);
    D.inv_cs_de_ef = (float)(1.0 / D.cs_de_e);
    D.inv_cs_de_if = (float)(1.0 / D.cs_de_i);
    D.ndt_ef = (float)(D.n_gas * D.dt_e);
    D.ndt_if = (float)(D.n_gas * D.dt_i);
    D.e_idx_ef = (float)(0.5 * kME / kQE / D.cs_de_e);
    D.g_idx_if = (float)(0.5 * mu_arar / kQE / D.cs_de_i);
    for (int s = 0; s < 2; ++s) {
        D.refl_eta[s] = p.refl_eta[s];
        D.see_gamma[s] = p.see_gamma[s];
        D.refl_etaf[s] = (float)p.refl_eta[s];
        D.see_gammaf[s] = (float)p.see_gamma[s];
    }
    D.see_sth = std::sqrt(p.see_te_ev * kQE / kME);
    D.see_sthf = (float)D.see_sth;
    D.inv_2dx = 1.0 / (2.0 * D.dx);
    D.edge_c = kQE * D.factor_w * 2.0 / 4294967296.0 * D.dx / (2.0 * kEPS0);
    D.ng = p.n_grid;
    D.nt = p.steps_per_cycle;
    D.nsub = p.ion_subcycle;
    D.n_harm = p.n_harmonics;
    D.eepf_bins = p.eepf_bins;
    D.ifed_bins = p.ifed_bins;
    D.cs_n_e = S->desc.size() > (size_t)d ? S->desc[d].cs_n_e : 1;
    D.cs_n_i = S->desc.size() > (size_t)d ? S->desc[d].cs_n_i : 1;
    D.active = 1;
    D.null_coll = p.null_collision;
    D.nxt = p.xt_bins;
    D.nbin = p.xt_bins > 0 ? p.steps_per_cycle / p.xt_bins : 0;
    D.stop_step = LLONG_MAX;
    D.cap[0] = p.capacity_e;
    D.cap[1] = p.capacity_i;
    D.seed = p.seed;
    for (int s = 0; s < 2; ++s) {
        D.x[s] = b + L.x[s];
        D.vx[s] = b + L.vx[s];
        D.vy[s] = b + L.vy[s];
        D.vz[s] = b + L.vz[s];
        // layout_of takes the four arrays one after another with the same padded size
        D.pstride[s] = (long long)(L.vx[s] - L.x[s]);
        D.holes[s] = reinterpret_cast<int *>(b + L.holes[s]);
    }
    D.q_e = reinterpret_cast<long long *>(b + L.q_e);
    D.q_i = reinterpret_cast<long long *>(b + L.q_i);
    D.acc_e = reinterpret_cast<long long *>(b + L.acc_e);
    D.acc_i = reinterpret_cast<long long *>(b + L.acc_i);
    D.n_e = reinterpret_cast<double *>(b + L.n_e);
    D.n_i = reinterpret_cast<double *>(b + L.n_i);
    D.phi = reinterpret_cast<double *>(b + L.phi);
    D.ef = reinterpret_cast<double *>(b + L.ef);
    D.ef_t = b + L.ef_t;
    D.f_cur = reinterpret_cast<long long *>(b + L.f_cur);
    D.fs = reinterpret_cast<FieldState *>(b + L.fs);
    D.sum_qe = reinterpret_cast<double *>(b + L.sum_qe);
    D.sum_qi = reinterpret_cast<double *>(b + L.sum_qi);
    D.sum_f = reinterpret_cast<double *>(b + L.sum_f);
    D.avg = reinterpret_cast<double *>(b + L.avg);
    D.eepf = reinterpret_cast<unsigned long long *>(b + L.eepf);
    D.ifed_pow = reinterpret_cast<unsigned long long *>(b + L.ifed_pow);
    D.ifed_gnd = reinterpret_cast<unsigned long long *>(b + L.ifed_gnd);
    D.power = reinterpret_cast<double *>(b + L.power);
    D.ctrl = S->d_ctrl + d;
    D.prod_parent = reinterpret_cast<int *>(b + L.prod_parent);
    D.sort_buf = reinterpret_cast<int *>(b + L.sort_buf);
    if (p.xt_bins > 0) {
        const size_t m = (size_t)p.n_grid * (size_t)p.xt_bins;
        double *x = reinterpret_cast<double *>(b + L.xt);
        D.xt_f = x;
        D.xt_qe = x + m;
        D.xt_qi = x + 2 * m;
        D.xt_cnti = x + 3 * m;
        D.xt_v[0] = x + 4 * m;
        D.xt_v[1] = x + 5 * m;
        D.xt_en[0] = x + 6 * m;
        D.xt_en[1] = x + 7 * m;
        D.xt_ion = x + 8 * m;
        D.xt_V = x + 9 * m;
        D.xt_d0 = D.xt_V + p.xt_bins;
        D.xt_steps = reinterpret_cast<long long *>(D.xt_d0 + p.xt_bins);
    }
    if (L.emit) {
        D.emit_parent = reinterpret_cast<int *>(b + L.emit_parent);
        D.emit_x = b + L.emit_x;
        for (int c = 0; c < 3; ++c) D.emit_v[c] = b + L.emit_v[c];
    }
    D.prod_x = b + L.prod_x;
    for (int c = 0; c < 3; ++c) {
        D.prod_ve[c] = b + L.prod_ve[c];
        D.prod_vi[c] = b + L.prod_vi[c];
    }
    for (int sp = 0; sp < 2; ++sp) {
        D.cs_sig[sp] = S->cs_sig[sp];
        D.cs_thr[sp] = S->cs_thr[sp];
        D.cs_max[sp] = S->cs_max[sp];
        D.cs_pm[sp] = S->cs_pm[sp];
        D.cs_shift[sp] = S->desc.size() > (size_t)d ? S->desc[d].cs_shift[sp] : 0;
    }
    D.lv_base = S->desc.size() > (size_t)d ? S->desc[d].lv_base : 0;
    D.lv_n = S->desc.size() > (size_t)d ? S->desc[d].lv_n : 1;
    D.vdrive = reinterpret_cast<const double *>(b + L.vdrive);
    D.sort_every = p.sort_every;
    if (p.sort_every > 0) {
        D.sort_cnt = reinterpret_cast<unsigned int *>(b + L.sort_cnt);
        for (int c = 0; c < 4; ++c) D.sort_tmp[c] = b + L.sort_tmp[c];
    }
    if (S->desc.size() <= (size_t)d) S->desc.resize(d + 1);
    S->desc[d] = D;
    null_bounds(S, d);
}

// Which push-kernel variant the species need: the null-collision one when
// an active discharge asks for the method.  Captured graphs carry the
// variant, so they are dropped when it changes.
void update_null_any(edupic_sim *S)
{
    int any[2] = {0, 0};
    for (int d = 0; d < S->nd && d < (int)S->desc.size(); ++d)
        if (S->desc[d].active)
            for (int sp = 0; sp < 2; ++sp) any[sp] |= (S->desc[d].null_coll >> sp) & 1;
    if (any[0] != S->null_any[0] || any[1] != S->null_any[1]) S->drop_graphs();
    S->null_any[0] = any[0];
    S->null_any[1] = any[1];
}

// Null-collision bound of discharge d from the host copy of the tables
// (Sec. 2.1.6): nu* = max_k (n sigma_tot,k) v_k with v_k the speed at the
// top of entry k's energy bin (energies round to the nearest entry), and
// P* = 1 - exp(-nu* dt).  Formed in the same order as the oracle's bound.
void null_bounds(edupic_sim *S, int d)
{
    DischargeDev &D = S->desc[d];
    // Bound of the Ar+ direct test (Algorithm 6).  An energy rounds to the
    // nearest entry k, so it lies below (k + 1/2) DE and the relative speed g
    // below v_k at that energy: n sigma_tot,k g <= n max_{k' <= k}(sigma_tot,k'
    // v_k'), the prefix maximum the kernel reads for the largest entry the ion
    // can reach.  The partner is drawn by Box-Muller, so its speed is at most
    // about 12.1 sigma_th (the largest normal the uniforms can give): g <=
    // |v| + 12.2 sigma_th.  Valid while that bound stays below the last
    // entry's speed (v2top); beyond it the full test is taken.
    for (int sp = 0; sp < 2; ++sp) {
        const double m = sp == 0 ? kME : kArMassU * kAMU / 2.0;
        const int n = S->sigsum_host[sp].empty() ? 0 : (int)S->sigsum_host[sp].size();
        const double vtop = n ? std::sqrt(2.0 * ((n - 0.5) * S->cs_de_host[sp]) * kQE / m) : 0.0;
        D.v2top[sp] = vtop * vtop * (1.0 - 1e-9);
        D.v2topf[sp] = (float)(vtop * vtop * (1.0 - 1e-5));
    }
    D.gcap = 12.2 * D.sig_th;
    D.gcapf = (float)(D.gcap * (1.0 + 1e-5));
    if (!D.null_coll) return;
    for (int sp = 0; sp < 2; ++sp) {
        const std::vector<double> &st = S->sigsum_host[sp];
        if (!((D.null_coll >> sp) & 1) || st.empty()) continue;
        const double m = sp == 0 ? kME : kArMassU * kAMU / 2.0;
        const double de = S->cs_de_host[sp];
        double best = 0.0;
        for (size_t k = 0; k < st.size(); ++k) {
            const double v = std::sqrt(2.0 * ((k + 0.5) * de) * kQE / m);
            const double nu = st[k] * D.n_gas * v;
            if (nu > best) best = nu;
        }
        const double dt = sp == 0 ? D.dt_e : D.dt_i;
        D.nu_star[sp] = best;
        D.p_star[sp] = 1.0 - std::exp(-best * dt);
        D.p_starf[sp] = (float)D.p_star[sp];
        D.null_ratf[sp] = best > 0.0 ? (float)(D.n_gas / best) : 0.0f;
    }
}

int upload_desc(edupic_sim *S)
{
    cudaError_t e = cudaMemcpyAsync(S->d_desc, S->desc.data(), sizeof(DischargeDev) * S->nd, cudaMemcpyHostToDevice,
                                    S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

int upload_desc_one(edupic_sim *S, int d)
{
    cudaError_t e = cudaMemcpyAsync(S->d_desc + d, &S->desc[d], sizeof(DischargeDev), cudaMemcpyHostToDevice,
                                    S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

void carve_shared(edupic_sim *S, int cs_entries)
{
    size_t o = 0;
    S->d_desc = reinterpret_cast<DischargeDev *>(S->arena);
    o = align_up(sizeof(DischargeDev) * S->nd, kAlign);
    S->d_ctrl = reinterpret_cast<Ctrl *>(S->arena + o);
    o += align_up(sizeof(Ctrl) * S->nd, kAlign);
    for (int sp = 0; sp < 2; ++sp) {
        S->cs_sig[sp] = S->arena + o;
        o += align_up((size_t)cs_entries * S->elem, kAlign);
    }
    for (int sp = 0; sp < 2; ++sp) {
        S->cs_thr[sp] = S->arena + o;
        o += align_up((size_t)cs_entries * 2 * S->elem, kAlign);
    }
    for (int sp = 0; sp < 2; ++sp) {
        S->cs_max[sp] = S->arena + o;
        o += align_up((size_t)kCoarse * S->elem, kAlign);
    }
    for (int sp = 0; sp < 2; ++sp) {
        S->cs_pm[sp] = S->arena + o;
        o += align_up((size_t)kCoarse * S->elem, kAlign);
    }
}

int setup_grid(edupic_sim *S)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EDUPIC_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::max(sms, 1);
    const bool f32 = S->precision == EDUPIC_FP32;
    for (int sp = 0; sp < 2; ++sp) {
        const int eb = sp == 0 ? S->eepf_max : 0;
        for (int sh = 0; sh < kPushShapeCount; ++sh) {
            const size_t smem = f32 ? Launch<float>::push_smem(S->nd, S->ng_max, eb, 0, sh)
                                    : Launch<double>::push_smem(S->nd, S->ng_max, eb, 0, sh);
            const int nb = f32 ? Launch<float>::push_blocks_per_sm(sp, smem, 0, sh)
                               : Launch<double>::push_blocks_per_sm(sp, smem, 0, sh);
            S->grid_shape[sp][sh] = std::max(nb, 0) * sms;
        }
        if (S->grid_shape[sp][0] < 1) return EDUPIC_ECUDA;  // the default shape must fit
        if (S->grid_shape[sp][S->shape[sp]] < 1) S->shape[sp] = 0;
        const size_t smem_xt = f32 ? Launch<float>::push_smem(S->nd, S->ng_max, eb, 1, 0)
                                   : Launch<double>::push_smem(S->nd, S->ng_max, eb, 1, 0);
        const int nb_xt = f32 ? Launch<float>::push_blocks_per_sm(sp, smem_xt, 1, 0)
                              : Launch<double>::push_blocks_per_sm(sp, smem_xt, 1, 0);
        if (nb_xt < 1 && S->xt_any) return EDUPIC_ECUDA;
        S->grid_xt[sp] = std::max(nb_xt, 0) * sms;
        S->grid[sp] = S->grid_max[sp] = S->grid_shape[sp][S->shape[sp]];
    }
    S->sms = sms;
    return EDUPIC_OK;
}

// The xt-accumulating kernel runs on the measured steps of a simulation that
// keeps xt diagnostics, on its own resident grid.
int xt_on(const edupic_sim *S, int measure) { return measure && S->xt_any ? 1 : 0; }
int push_grid(const edupic_sim *S, int sp, int measure) { return xt_on(S, measure) ? S->grid_xt[sp] : S->grid[sp]; }

template <typename T>
int launch_step(edupic_sim *S, bool ion, int measure)
{
    cudaError_t e = Launch<T>::push(S->d_desc, S->nd, 0, measure, push_grid(S, 0, measure), S->ng_max,
                                    S->eepf_max, S->null_any[0], xt_on(S, measure), S->shape[0], S->sort_any, S->stream);
    if (e == cudaSuccess && ion)
        e = Launch<T>::push(S->d_desc, S->nd, 1, measure, push_grid(S, 1, measure), S->ng_max,
                            S->eepf_max, S->null_any[1], xt_on(S, measure), S->shape[1], S->sort_any, S->stream);
    if (e == cudaSuccess) e = Launch<T>::finalize(S->d_desc, S->nd, ion ? 1 : 0, measure, S->stream);
    return cuda_status(e);
}

cudaError_t launch_sort(edupic_sim *S);

// One time step; `last` (the final step of an ion subcycle) adds the periodic
// cell sort, which every discharge decides on from its own step count.
int launch_one(edupic_sim *S, bool ion, int measure, bool last)
{
    int rc = S->precision == EDUPIC_FP32 ? launch_step<float>(S, ion, measure) : launch_step<double>(S, ion, measure);
    if (rc == EDUPIC_OK && last && S->sort_any) rc = cuda_status(launch_sort(S));
    return rc;
}

cudaError_t launch_sort(edupic_sim *S)
{
    return S->precision == EDUPIC_FP32 ? Launch<float>::sort(S->d_desc, S->nd, S->ng_max, S->sms, S->stream)
                                       : Launch<double>::sort(S->d_desc, S->nd, S->ng_max, S->sms, S->stream);
}

// One ion subcycle (N_SUB steps starting at phase 0) as a CUDA graph.
int build_graph(edupic_sim *S, int measure)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return EDUPIC_ECUDA;
    int rc = EDUPIC_OK;
    for (int k = 0; k < S->nsub && rc == EDUPIC_OK; ++k) rc = launch_one(S, k == 0, measure, k == S->nsub - 1);
    e = cudaStreamEndCapture(S->stream, &g);
    if (rc != EDUPIC_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return EDUPIC_ECUDA;
    }
    e = cudaGraphInstantiate(&S->graph[measure], g, 0);
    cudaGraphDestroy(g);
    return cuda_status(e);
}

int read_ctrl(edupic_sim *S, int d, Ctrl *c)
{
    cudaError_t e = cudaStreamSynchronize(S->stream);
    if (e == cudaSuccess) e = cudaMemcpy(c, S->ctrl(d), sizeof(Ctrl), cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

int error_of(const Ctrl &c)
{
    if (c.error & kErrNan) return EDUPIC_ENAN;
    if (c.error & kErrTimeout) return EDUPIC_ETIMEOUT;
    if (c.error) return EDUPIC_ECAPACITY;
    return EDUPIC_OK;
}

// Bucket of v^2 as the particle kernel forms it (lv_bucket): exponent and top
// five mantissa bits of the particle-precision value, and the smallest v^2 of
// a bucket.
static uint64_t lv_bits(float w2)
{
    uint32_t b;
    std::memcpy(&b, &w2, 4);
    return b >> 18;
}
static uint64_t lv_bits(double w2)
{
    uint64_t b;
    std::memcpy(&b, &w2, 8);
    return b >> 47;
}
template <typename T>
static T lv_lower(uint64_t j)
{
    T w;
    if constexpr (sizeof(T) == 4) {
        const uint32_t b = (uint32_t)(j << 18);
        std::memcpy(&w, &b, 4);
    } else {
        const uint64_t b = j << 47;
        std::memcpy(&w, &b, 8);
    }
    return w;
}

// The electrons' collision bound per v^2 bucket (replaces the coarse table of
// species 0): for each bucket, the largest sigma_tot,k over every entry k the
// kernel's nearest-entry index can take for a v^2 in the bucket (one entry of
// margin on each side for the rounding of the index arithmetic) times the
// speed at the bucket's top, widened by 1e-6 and rounded up.  The kernel
// multiplies by n dt: P_coll = 1 - exp(-n sigma_tot v dt) of any particle in
// the bucket lies below it.  Buckets above the table's last entry (where the
// clamped entry meets unbounded speeds) and the last bucket are +inf.
template <typename T>
void lv_table(const std::vector<T> &sum, double de_ev, std::vector<T> &out, int &base, int &nbuckets)
{
    const int n = (int)sum.size();
    // the entry index of v^2 as the kernel forms it (FP32: v^2 * s + 0.5 with
    // s rounded to float; FP64: (m/2) v^2 / e / de + 0.5), before the clamp
    const double sf = (double)(float)(0.5 * kME / kQE / de_ev);
    auto kidx = [&](double w2) -> long long {
        const double r = sizeof(T) == 4 ? w2 * sf + 0.5 : 0.5 * kME * w2 / kQE / de_ev + 0.5;
        return r >= 4e18 ? (long long)4e18 : (long long)std::floor(r);
    };
    // top: a v^2 whose entry is past the last one
    const double w2_top = (sizeof(T) == 4 ? (n + 1.0) / sf : (n + 1.0) * de_ev * kQE / (0.5 * kME));
    const uint64_t jt = lv_bits((T)w2_top) + 1;          // unbounded from this bucket on
    const uint64_t j0 = jt >= (uint64_t)(kCoarse - 1) ? jt - (kCoarse - 1) : 0;
    const int nb = (int)(jt - j0 + 1);
    out.assign(kCoarse, (T)INFINITY);
    for (int j = 0; j + 1 < nb; ++j) {
        const double lo = j == 0 ? 0.0 : (double)lv_lower<T>(j0 + j);
        const double hi = (double)lv_lower<T>(j0 + j + 1);
        const long long a = std::max(0ll, kidx(lo) - 1), b = std::min((long long)n - 1, kidx(hi) + 1);
        double m = 0.0;
        for (long long k = a; k <= b; ++k) m = std::max(m, (double)sum[(size_t)k]);
        const double v = m * std::sqrt(hi) * (1.0 + 1e-6);
        T t = (T)v;
        if ((double)t < v) t = std::nextafter(t, (T)INFINITY);
        out[(size_t)j] = t;
    }
    base = (int)j0;
    nbuckets = nb;
}

template <typename T>
int upload_tables(edupic_sim *S, int species, int n_proc, int n_entries, double de_ev, const double *sig)
{
    std::vector<T> sum((size_t)n_entries);
    std::vector<T> thr(2 * (size_t)n_entries);
    for (int k = 0; k < n_entries; ++k) {
        const double s0 = sig[k], s1 = sig[(size_t)n_entries + k];
        const double s2 = n_proc == 3 ? sig[2 * (size_t)n_entries + k] : 0.0;
        // the processes summed in their order (elastic, excitation, ionisation)
        const double stot = n_proc == 3 ? s0 + s1 + s2 : s0 + s1;
        sum[k] = (T)stot;
        thr[2 * (size_t)k] = (T)(s0 / stot);
        thr[2 * (size_t)k + 1] = (T)(n_proc == 3 ? (s0 + s1) / stot : 1.0);
    }
    // coarse maxima over 2^shift entries: an upper bound of n*sigma_tot used to
    // skip the fine lookup when R01 lies above the bound's probability
    int shift = 0;
    while (((n_entries - 1) >> shift) >= kCoarse) ++shift;
    std::vector<T> cmax(kCoarse, (T)0);
    for (int k = 0; k < n_entries; ++k) {
        const int j = k >> shift;
        const double v = (double)sum[k] * (1.0 + 1e-6);
        T t = (T)v;
        if ((double)t < v) t = std::nextafter(t, (T)INFINITY);
        if (t > cmax[j]) cmax[j] = t;
    }
    // prefix maxima of sigma_tot,k * v_k (v_k the lab / relative speed at the
    // top of entry k's energy bin) up to the end of each coarse block: a bound
    // of sigma_tot * g over every energy up to that block (rounded up)
    std::vector<T> pmax(kCoarse, (T)0);
    {
        const double m = species == 0 ? kME : 0.5 * kArMassU * kAMU;
        double run = 0.0;
        for (int k = 0; k < n_entries; ++k) {
            run = std::max(run, (double)sum[k] * std::sqrt(2.0 * ((k + 0.5) * de_ev) * kQE / m));
            const int j = k >> shift;
            const double v = run * (1.0 + 1e-6);
            T t = (T)v;
            if ((double)t < v) t = std::nextafter(t, (T)INFINITY);
            pmax[j] = t;  // the last entry of block j leaves the block's prefix maximum
        }
        for (int j = ((n_entries - 1) >> shift) + 1; j < kCoarse; ++j) pmax[j] = pmax[j - 1];
    }
    S->cs_shift_pending[species] = shift;
    if (species == 0) lv_table<T>(sum, de_ev, cmax, S->lv_base_pending, S->lv_n_pending);
    cudaError_t e = cudaMemcpyAsync(S->cs_max[species], cmax.data(), sizeof(T) * kCoarse, cudaMemcpyHostToDevice,
                                    S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->cs_pm[species], pmax.data(), sizeof(T) * kCoarse, cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->cs_sig[species], sum.data(), sizeof(T) * sum.size(), cudaMemcpyHostToDevice,
                            S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->cs_thr[species], thr.data(), sizeof(T) * thr.size(), cudaMemcpyHostToDevice,
                            S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

// Drive voltage at the N_T steps of one RF cycle, V(t) = sum V_k cos(2 pi f_k t)
// with t = step * dt_e (the waveform input of the field solve).
int upload_drive(edupic_sim *S, int d)
{
    const edupic_params &p = S->params[d];
    const double dt_e = S->desc[d].dt_e, pi = 3.14159265358979323846;
    const double bias = (size_t)d < S->v_bias.size() ? S->v_bias[(size_t)d] : 0.0;
    std::vector<double> v((size_t)p.steps_per_cycle);
    for (int tc = 0; tc < p.steps_per_cycle; ++tc) {
        const double t = (double)tc * dt_e;
        double a = 0.0;
        for (int h = 0; h < p.n_harmonics; ++h) a += p.harm_volt_v[h] * std::cos(2.0 * pi * p.harm_freq_hz[h] * t);
        v[tc] = a + bias;
    }
    cudaError_t e = cudaMemcpyAsync(const_cast<double *>(S->desc[d].vdrive), v.data(), sizeof(double) * v.size(),
                                    cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

// A fixed team of host threads for the particle conversions, created on first
// use (up to 16 with the calling thread) and kept for the process.  One run
// at a time; run(nt, f) calls f(t) for t = 0..nt-1, t = 0 on the caller.
class HostTeam {
public:
    static HostTeam &get()
    {
        static HostTeam team;
        return team;
    }
    int size() const { return (int)workers_.size() + 1; }
    void run(int nt, const std::function<void(int)> &f)
    {
        std::lock_guard<std::mutex> serial(run_mutex_);
        {
            std::lock_guard<std::mutex> lk(m_);
            job_ = &f;
            n_ = nt;
            left_ = nt - 1;
            ++gen_;
        }
        cv_.notify_all();
        f(0);
        std::unique_lock<std::mutex> lk(m_);
        done_.wait(lk, [&] { return left_ == 0; });
        job_ = nullptr;
    }
    ~HostTeam()
    {
        {
            std::lock_guard<std::mutex> lk(m_);
            stop_ = true;
            ++gen_;
        }
        cv_.notify_all();
        for (auto &w : workers_) w.join();
    }

private:
    HostTeam()
    {
        const int hw = std::max(1, (int)std::thread::hardware_concurrency());
        for (int i = 1; i < std::min(hw, 16); ++i) workers_.emplace_back([this, i] { loop(i); });
    }
    void loop(int id)
    {
        unsigned long long seen = 0;
        for (;;) {
            const std::function<void(int)> *f;
            int n;
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
                f = job_;
                n = n_;
            }
            if (id < n) {  // a run does not end before its workers report, so none is missed
                (*f)(id);
                std::lock_guard<std::mutex> lk(m_);
                if (--left_ == 0) done_.notify_one();
            }
        }
    }
    std::vector<std::thread> workers_;
    std::mutex run_mutex_, m_;
    std::condition_variable cv_, done_;
    const std::function<void(int)> *job_ = nullptr;
    int n_ = 0, left_ = 0;
    unsigned long long gen_ = 0;
    bool stop_ = false;
};

// Run f(lo, hi) over [0, n) on the host team (ranges of at least 64 Ki
// elements; small n runs on the calling thread).
template <typename F>
void parallel_ranges(int64_t n, F f)
{
    constexpr int64_t kGrain = 1 << 16;
    const int64_t chunks = (n + kGrain - 1) / kGrain;
    if (chunks <= 1) {
        f((int64_t)0, n);
        return;
    }
    HostTeam &team = HostTeam::get();
    const int nt = (int)std::min<int64_t>(team.size(), chunks);
    team.run(nt, [&](int t) { f(n * t / nt, n * (t + 1) / nt); });
}

// Page-locked host staging buffer of the object (grown on demand, freed with it).
void *pinned_reserve(edupic_sim *S, size_t bytes)
{
    if (S->pinned_bytes >= bytes) return S->pinned;
    if (S->pinned) cudaFreeHost(S->pinned);
    S->pinned = nullptr;
    S->pinned_bytes = 0;
    void *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) return nullptr;
    S->pinned = p;
    S->pinned_bytes = bytes;
    return p;
}

// x, vx, vy, vz checked (0 <= x <= L, finite velocities; a value v is finite
// when v - v == 0) and converted to T in one parallel pass into the pinned
// stage, arrays one after another.  Loops without branches, so that they
// vectorise.
template <typename T>
int convert_stage(edupic_sim *S, int d, int64_t n, const double *const src[4], T *stage)
{
    const double L = S->params[d].gap_m;
    std::atomic<int> bad{0};
    parallel_ranges(n, [&](int64_t lo, int64_t hi) {
        int b = 0;
        {
            const double *x = src[0];
            T *o = stage;
            for (int64_t j = lo; j < hi; ++j) {
                const double v = x[j];
                o[j] = (T)v;
                b |= (int)!(v >= 0.0) | (int)!(v <= L);
            }
        }
        for (int c = 1; c < 4; ++c) {
            const double *v = src[c];
            T *o = stage + (size_t)c * (size_t)n;
            for (int64_t j = lo; j < hi; ++j) {
                const double a = v[j];
                o[j] = (T)a;
                b |= (int)!(a - a == 0.0);
            }
        }
        if (b) bad.store(1, std::memory_order_relaxed);
    });
    return bad.load() ? EDUPIC_EINVAL : EDUPIC_OK;
}

// The same checks without conversion: true when every value is acceptable.
bool particles_valid(edupic_sim *S, int d, int64_t n, const double *const src[4])
{
    const double L = S->params[d].gap_m;
    std::atomic<int> bad{0};
    parallel_ranges(n, [&](int64_t lo, int64_t hi) {
        int b = 0;
        for (int64_t j = lo; j < hi; ++j) {
            const double v = src[0][j];
            b |= (int)!(v >= 0.0) | (int)!(v <= L);
        }
        for (int c = 1; c < 4; ++c)
            for (int64_t j = lo; j < hi; ++j) {
                const double a = src[c][j];
                b |= (int)!(a - a == 0.0);
            }
        if (b) bad.store(1, std::memory_order_relaxed);
    });
    return bad.load() == 0;
}

template <typename T>
int download_particles(edupic_sim *S, int d, int sp, int64_t n, double *const dst[4])
{
    const void *src[4] = {S->desc[d].x[sp], S->desc[d].vx[sp], S->desc[d].vy[sp], S->desc[d].vz[sp]};
    std::vector<T> tmp((size_t)n);
    for (int c = 0; c < 4; ++c) {
        if (!dst[c]) continue;
        cudaError_t e = cudaMemcpy(tmp.data(), src[c], sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return EDUPIC_ECUDA;
        for (int64_t j = 0; j < n; ++j) dst[c][j] = (double)tmp[j];
    }
    return EDUPIC_OK;
}

// Replace the particles of species sp of discharge d (Algorithm 1's
// initialisation, or a reload): check and convert the host arrays into the
// pinned stage, copy them and the count, and form the densities and the field
// of the current step again.  One synchronisation, as the stage is reused by
// the next load.
int load_species(edupic_sim *S, int d, int sp, int64_t n, const double *const src[4])
{
    const size_t body = align_up(4 * S->elem * (size_t)n, 16);
    unsigned char *stage = static_cast<unsigned char *>(pinned_reserve(S, body + 16));
    if (!stage) return EDUPIC_ENOMEM;
    const DischargeDev &D = S->desc[d];
    void *dst[4] = {D.x[sp], D.vx[sp], D.vy[sp], D.vz[sp]};
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        const int rc = S->precision == EDUPIC_FP32
                           ? convert_stage<float>(S, d, n, src, reinterpret_cast<float *>(stage))
                           : convert_stage<double>(S, d, n, src, reinterpret_cast<double *>(stage));
        if (rc) return rc;
        for (int c = 0; c < 4 && e == cudaSuccess; ++c)
            e = cudaMemcpyAsync(dst[c], stage + (size_t)c * S->elem * (size_t)n, S->elem * (size_t)n,
                                cudaMemcpyHostToDevice, S->stream);
    }
    long long *count = reinterpret_cast<long long *>(stage + body);
    *count = n;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&S->ctrl(d)->n[sp], count, sizeof(long long), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) e = enqueue_refresh(S, d, sp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

// Densities of species sp of discharge d from its particles, and the field
// of the current step, queued on the stream.
cudaError_t enqueue_refresh(edupic_sim *S, int d, int sp)
{
    const DischargeDev &D = S->desc[d];
    cudaError_t e = cudaSuccess;
    const size_t ng = (size_t)S->params[d].n_grid;
    if (e == cudaSuccess) e = cudaMemsetAsync(sp == 0 ? D.q_e : D.q_i, 0, ng * 8, S->stream);
    if (e == cudaSuccess && sp == 1) e = cudaMemsetAsync(D.acc_i, 0, ng * 8, S->stream);
    const int also_acc = (sp == 1 && S->phase != 0) ? 1 : 0;
    if (e == cudaSuccess)
        e = S->precision == EDUPIC_FP32 ? Launch<float>::deposit(S->d_desc, S->nd, d, sp, also_acc, S->stream)
                                        : Launch<double>::deposit(S->d_desc, S->nd, d, sp, also_acc, S->stream);
    if (e == cudaSuccess)
        e = S->precision == EDUPIC_FP32 ? Launch<float>::fields(S->d_desc, S->nd, d, S->stream)
                                        : Launch<double>::fields(S->d_desc, S->nd, d, S->stream);
    return e;
}

bool valid_d(const edupic_sim *S, int d) { return S && d >= 0 && d < S->nd; }

}  // namespace host
}  // namespace edupic

extern "C" {

int edupic_arena_bytes(int nd, const edupic_params *params, int precision, size_t *bytes)
{
    int rc = check_params(nd, params, precision);
    if (rc) return rc;
    if (!bytes) return EDUPIC_EINVAL;
    const size_t elem = precision == EDUPIC_FP32 ? 4 : 8;
    size_t tot = shared_bytes(nd, elem, params[0].cs_entries);
    for (int d = 0; d < nd; ++d) tot += layout_of(params[d], elem).bytes;
    *bytes = tot;
    return EDUPIC_OK;
}

int edupic_create(int nd, const edupic_params *params, int precision, void *device_arena, size_t arena_bytes,
                  void *cuda_stream, edupic_sim **out)
{
    if (!out) return EDUPIC_EINVAL;
    *out = nullptr;
    size_t need = 0;
    int rc = edupic_arena_bytes(nd, params, precision, &need);
    if (rc) return rc;
    if (!device_arena || ((uintptr_t)device_arena % kAlign)) return EDUPIC_EINVAL;
    if (arena_bytes < need) return EDUPIC_ENOMEM;
    edupic_sim *S = new (std::nothrow) edupic_sim();
    if (!S) return EDUPIC_ENOMEM;
    S->nd = nd;
    S->precision = precision;
    S->elem = precision == EDUPIC_FP32 ? 4 : 8;
    S->params.assign(params, params + nd);
    S->v_bias.assign((size_t)nd, 0.0);
    S->arena = static_cast<unsigned char *>(device_arena);
    S->arena_bytes = arena_bytes;
    S->stream = static_cast<cudaStream_t>(cuda_stream);
    S->nsub = params[0].ion_subcycle;
    S->nt_common = params[0].steps_per_cycle;
    for (int d = 0; d < nd; ++d) {
        S->ng_max = std::max(S->ng_max, params[d].n_grid);
        S->eepf_max = std::max(S->eepf_max, params[d].eepf_bins);
        if (params[d].steps_per_cycle != S->nt_common) S->nt_common = -1;
    }
    // shared region: descriptors, packed controls, the two cross-section tables
    carve_shared(S, params[0].cs_entries);
    size_t o = shared_bytes(nd, S->elem, params[0].cs_entries);
    for (int d = 0; d < nd; ++d) {
        S->layouts.push_back(layout_of(params[d], S->elem));
        S->base.push_back(o);
        o += S->layouts.back().bytes;
    }
    for (int d = 0; d < nd; ++d) fill_desc(S, d);
    update_null_any(S);
    for (int d = 0; d < nd; ++d) S->xt_any |= params[d].xt_bins > 0 ? 1 : 0;
    for (int d = 0; d < nd; ++d) S->sort_any |= params[d].sort_every > 0 ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(S->arena, 0, need, S->stream);
    if (e != cudaSuccess) {
        delete S;
        return EDUPIC_ECUDA;
    }
    rc = upload_desc(S);
    for (int d = 0; d < nd && rc == EDUPIC_OK; ++d) rc = upload_drive(S, d);
    if (rc) {
        delete S;
        return rc;
    }
    rc = setup_grid(S);
    if (rc) {
        delete S;
        return rc;
    }
    // the field of step 0 (empty discharge: the vacuum field of V(0))
    for (int d = 0; d < nd && rc == EDUPIC_OK; ++d) {
        e = precision == EDUPIC_FP32 ? Launch<float>::fields(S->d_desc, nd, d, S->stream)
                                     : Launch<double>::fields(S->d_desc, nd, d, S->stream);
        rc = cuda_status(e);
    }
    if (rc == EDUPIC_OK) rc = cuda_status(cudaStreamSynchronize(S->stream));
    if (rc) {
        delete S;
        return rc;
    }
    *out = S;
    return EDUPIC_OK;
}

int edupic_destroy(edupic_sim *S)
{
    if (!S) return EDUPIC_EINVAL;
    if (S->stream) cudaStreamSynchronize(S->stream);
    delete S;
    return EDUPIC_OK;
}

int edupic_electron_bound_table(int precision, int n_entries, double de_ev, const double *sigma_sum,
                                double *table_out, int *base_out, int *n_out)
{
    if (!sigma_sum || !table_out || !base_out || !n_out || n_entries < 1 || !(de_ev > 0) ||
        (precision != EDUPIC_FP32 && precision != EDUPIC_FP64))
        return EDUPIC_EINVAL;
    static_assert(EDUPIC_BOUND_BUCKETS == kCoarse, "the header states the table's length");
    for (int k = 0; k < n_entries; ++k)
        if (!(sigma_sum[k] >= 0) || !std::isfinite(sigma_sum[k])) return EDUPIC_EINVAL;
    auto run = [&](auto zero) {
        using T = decltype(zero);
        std::vector<T> sum((size_t)n_entries), out;
        for (int k = 0; k < n_entries; ++k) sum[(size_t)k] = (T)sigma_sum[k];
        lv_table<T>(sum, de_ev, out, *base_out, *n_out);
        for (int j = 0; j < kCoarse; ++j) table_out[j] = (double)out[(size_t)j];
    };
    if (precision == EDUPIC_FP32)
        run(0.0f);
    else
        run(0.0);
    return EDUPIC_OK;
}

int edupic_set_cross_sections(edupic_sim *S, int species, int n_proc, int n_entries, double de_ev,
                              const double *sigma_m2)
{
    if (!S || !sigma_m2 || (species != 0 && species != 1) || !(de_ev > 0)) return EDUPIC_EINVAL;
    if ((species == 0 && n_proc != 3) || (species == 1 && n_proc != 2)) return EDUPIC_EINVAL;
    if (n_entries < 1 || n_entries > S->params[0].cs_entries) return EDUPIC_EINVAL;
    for (size_t k = 0; k < (size_t)n_proc * n_entries; ++k)
        if (!(sigma_m2[k] >= 0) || !std::isfinite(sigma_m2[k])) return EDUPIC_EINVAL;
    int rc = S->precision == EDUPIC_FP32 ? upload_tables<float>(S, species, n_proc, n_entries, de_ev, sigma_m2)
                                         : upload_tables<double>(S, species, n_proc, n_entries, de_ev, sigma_m2);
    if (rc) return rc;
    for (int d = 0; d < S->nd; ++d) {
        S->desc[d].cs_shift[species] = S->cs_shift_pending[species];
        if (species == 0) {
            S->desc[d].lv_base = S->lv_base_pending;
            S->desc[d].lv_n = S->lv_n_pending;
            S->desc[d].cs_n_e = n_entries;
            S->desc[d].cs_de_e = de_ev;
            S->desc[d].inv_cs_de_ef = (float)(1.0 / de_ev);
            S->desc[d].e_idx_ef = (float)(0.5 * kME / kQE / de_ev);
        } else {
            S->desc[d].cs_n_i = n_entries;
            S->desc[d].cs_de_i = de_ev;
            S->desc[d].inv_cs_de_if = (float)(1.0 / de_ev);
            S->desc[d].g_idx_if = (float)(0.5 * (kArMassU * kAMU / 2.0) / kQE / de_ev);
        }
    }
    // largest sigma_tot * v of the table (v of the lookup energy: e- lab
    // speed, Ar+ relative speed with the reduced mass), for the accuracy check
    {
        const double m = species == 0 ? kME : 0.5 * kArMassU * kAMU;
        double best = 0.0;
        for (int k = 0; k < n_entries; ++k) {
            double st = 0.0;
            for (int q = 0; q < n_proc; ++q) st += sigma_m2[(size_t)q * n_entries + k];
            const double v = std::sqrt(2.0 * (k * de_ev) * kQE / m);
            best = std::max(best, st * v);
        }
        S->sigv_max[species] = best;
    }
    S->sigsum_host[species].resize((size_t)n_entries);
    double top = 0.0;
    for (int k = 0; k < n_entries; ++k) {
        // processes summed in order from zero, as the collision test's table
        double st = 0.0;
        for (int q = 0; q < n_proc; ++q) st += sigma_m2[(size_t)q * n_entries + k];
        S->sigsum_host[species][(size_t)k] = st;
        const double m = species == 0 ? kME : 0.5 * kArMassU * kAMU;
        top = std::max(top, st * std::sqrt(2.0 * ((k + 0.5) * de_ev) * kQE / m));
    }
    S->sigv_top[species] = top;
    S->cs_de_host[species] = de_ev;
    for (int d = 0; d < S->nd; ++d) null_bounds(S, d);
    S->cs_set[species] = true;
    return upload_desc(S);
}

int edupic_load_particles(edupic_sim *S, int d, int species, int64_t n, const double *x, const double *vx,
                          const double *vy, const double *vz)
{
    if (!valid_d(S, d) || (species != 0 && species != 1) || n < 0) return EDUPIC_EINVAL;
    if (n > (species == 0 ? S->params[d].capacity_e : S->params[d].capacity_i)) return EDUPIC_ECAPACITY;
    if (n > 0 && (!x || !vx || !vy || !vz)) return EDUPIC_EINVAL;
    const double *src[4] = {x, vx, vy, vz};  // checked while they are converted
    return load_species(S, d, species, n, src);
}

int edupic_seed(edupic_sim *S, int d, int64_t n_init)
{
    if (!valid_d(S, d) || n_init < 0) return EDUPIC_EINVAL;
    if (n_init > S->params[d].capacity_e || n_init > S->params[d].capacity_i) return EDUPIC_ECAPACITY;
    cudaError_t e = cudaSuccess;
    for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp) {
        e = S->precision == EDUPIC_FP32 ? Launch<float>::seed(S->d_desc, d, sp, n_init, S->stream)
                                        : Launch<double>::seed(S->d_desc, d, sp, n_init, S->stream);
        if (e == cudaSuccess) e = enqueue_refresh(S, d, sp);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

int edupic_step(edupic_sim *S, int64_t n_steps, int measure)
{
    if (!S || n_steps < 0) return EDUPIC_EINVAL;
    if (!S->cs_set[0] || !S->cs_set[1]) return EDUPIC_ESTATE;
    measure = measure ? 1 : 0;
    const bool can_graph = S->graphs && S->stream != nullptr;
    int64_t i = 0;
    while (i < n_steps) {
        if (can_graph && S->phase == 0 && n_steps - i >= S->nsub) {
            if (!S->graph[measure]) {
                int rc = build_graph(S, measure);
                if (rc) return rc;
            }
            cudaError_t e = cudaGraphLaunch(S->graph[measure], S->stream);
            if (e != cudaSuccess) return EDUPIC_ECUDA;
            i += S->nsub;
            continue;
        }
        int rc = launch_one(S, S->phase == 0, measure, S->phase == S->nsub - 1);
        if (rc) return rc;
        S->phase = (S->phase + 1) % S->nsub;
        ++i;
    }
    return EDUPIC_OK;
}

int edupic_run_cycles(edupic_sim *S, int n_cycles, int measure)
{
    if (!S || n_cycles < 0) return EDUPIC_EINVAL;
    if (S->nt_common < 0) return EDUPIC_EINVAL;
    return edupic_step(S, (int64_t)n_cycles * S->nt_common, measure);
}

int edupic_synchronize(edupic_sim *S)
{
    if (!S) return EDUPIC_EINVAL;
    if (cudaStreamSynchronize(S->stream) != cudaSuccess) return EDUPIC_ECUDA;
    for (int d = 0; d < S->nd; ++d) {
        Ctrl c;
        int rc = read_ctrl(S, d, &c);
        if (rc) return rc;
        rc = error_of(c);
        if (rc) return rc;
    }
    return EDUPIC_OK;
}

int edupic_selftest_wait_expiry(edupic_sim *S, int d, int64_t limit_ns)
{
    if (!valid_d(S, d) || limit_ns < 1000 || limit_ns > (int64_t)kWaitLimitNs) return EDUPIC_EINVAL;
    int *err = &S->ctrl(d)->error;
    cudaError_t e = S->precision == EDUPIC_FP32 ? Launch<float>::wait_expiry((unsigned long long)limit_ns, err, S->stream)
                                                : Launch<double>::wait_expiry((unsigned long long)limit_ns, err, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) return EDUPIC_ECUDA;
    Ctrl c;
    int rc = read_ctrl(S, d, &c);
    return rc ? rc : error_of(c);
}

int edupic_profile_steps(edupic_sim *S, int64_t n_steps, int measure, double out_ms[3], int64_t launches[3])
{
    if (!S || n_steps < 0 || !out_ms || !launches) return EDUPIC_EINVAL;
    if (!S->cs_set[0] || !S->cs_set[1]) return EDUPIC_ESTATE;
    measure = measure ? 1 : 0;
    for (int k = 0; k < 3; ++k) {
        out_ms[k] = 0.0;
        launches[k] = 0;
    }
    // all steps are enqueued back to back, with an event pair around every
    // kernel, and read after one synchronisation
    constexpr int64_t kChunk = 256;
    std::vector<cudaEvent_t> ev(4 * kChunk);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return EDUPIC_ECUDA;
    int rc = EDUPIC_OK;
    for (int64_t done = 0; done < n_steps && rc == EDUPIC_OK;) {
        const int64_t m = std::min<int64_t>(kChunk, n_steps - done);
        std::vector<char> ion(m);
        cudaError_t e = cudaSuccess;
        for (int64_t i = 0; i < m && e == cudaSuccess; ++i) {
            ion[i] = S->phase == 0;
            cudaEvent_t *E = &ev[4 * i];
            e = cudaEventRecord(E[0], S->stream);
            if (S->precision == EDUPIC_FP32) {
                if (e == cudaSuccess)
                    e = Launch<float>::push(S->d_desc, S->nd, 0, measure, push_grid(S, 0, measure), S->ng_max,
                                            S->eepf_max, S->null_any[0], xt_on(S, measure), S->shape[0], S->sort_any, S->stream);
                if (e == cudaSuccess) e = cudaEventRecord(E[1], S->stream);
                if (e == cudaSuccess && ion[i])
                    e = Launch<float>::push(S->d_desc, S->nd, 1, measure, push_grid(S, 1, measure), S->ng_max,
                                            S->eepf_max, S->null_any[1], xt_on(S, measure), S->shape[1], S->sort_any, S->stream);
                if (e == cudaSuccess) e = cudaEventRecord(E[2], S->stream);
                if (e == cudaSuccess) e = Launch<float>::finalize(S->d_desc, S->nd, ion[i], measure, S->stream);
            } else {
                if (e == cudaSuccess)
                    e = Launch<double>::push(S->d_desc, S->nd, 0, measure, push_grid(S, 0, measure), S->ng_max,
                                            S->eepf_max, S->null_any[0], xt_on(S, measure), S->shape[0], S->sort_any, S->stream);
                if (e == cudaSuccess) e = cudaEventRecord(E[1], S->stream);
                if (e == cudaSuccess && ion[i])
                    e = Launch<double>::push(S->d_desc, S->nd, 1, measure, push_grid(S, 1, measure), S->ng_max,
                                            S->eepf_max, S->null_any[1], xt_on(S, measure), S->shape[1], S->sort_any, S->stream);
                if (e == cudaSuccess) e = cudaEventRecord(E[2], S->stream);
                if (e == cudaSuccess) e = Launch<double>::finalize(S->d_desc, S->nd, ion[i], measure, S->stream);
            }
            if (e == cudaSuccess && S->sort_any && S->phase == S->nsub - 1) e = launch_sort(S);
            if (e == cudaSuccess) e = cudaEventRecord(E[3], S->stream);
            S->phase = (S->phase + 1) % S->nsub;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        for (int64_t i = 0; i < m && e == cudaSuccess; ++i) {
            const cudaEvent_t *E = &ev[4 * i];
            float ms[3] = {0, 0, 0};
            e = cudaEventElapsedTime(&ms[0], E[0], E[1]);
            if (e == cudaSuccess && ion[i]) e = cudaEventElapsedTime(&ms[1], E[1], E[2]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[2], E[2], E[3]);
            out_ms[0] += ms[0];
            out_ms[1] += ms[1];
            out_ms[2] += ms[2];
            launches[0] += 1;
            launches[1] += ion[i] ? 1 : 0;
            launches[2] += 1;
        }
        if (e != cudaSuccess) rc = EDUPIC_ECUDA;
        done += m;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

int edupic_set_push_grid(edupic_sim *S, int species, int blocks)
{
    if (!S || (species != 0 && species != 1) || blocks < 0) return EDUPIC_EINVAL;
    // only the resident limit: persistent grids below it (with kernel
    // versions since withdrawn) stalled on a 64-discharge batch without a
    // cause found, so such grids are refused
    if (blocks != 0 && blocks != S->grid_max[species]) return EDUPIC_EINVAL;
    const int g = S->grid_max[species];
    if (g != S->grid[species]) {
        S->grid[species] = g;
        S->drop_graphs();  // captured launches carry the grid
    }
    return EDUPIC_OK;
}

int edupic_get_push_grid(edupic_sim *S, int out[2])
{
    if (!S || !out) return EDUPIC_EINVAL;
    out[0] = S->grid[0];
    out[1] = S->grid[1];
    return EDUPIC_OK;
}

// Make shape sh the particle kernel's launch shape for species sp.
static void select_shape(edupic_sim *S, int sp, int sh)
{
    if (S->shape[sp] == sh && S->grid[sp] == S->grid_shape[sp][sh]) return;
    S->shape[sp] = sh;
    S->grid[sp] = S->grid_max[sp] = S->grid_shape[sp][sh];
    S->drop_graphs();  // captured launches carry the shape and grid
}

int edupic_set_push_shape(edupic_sim *S, int species, int shape)
{
    if (!S || (species != 0 && species != 1) || shape < 0 || shape >= kPushShapeCount) return EDUPIC_EINVAL;
    if (S->grid_shape[species][shape] < 1) return EDUPIC_EINVAL;  // does not fit this object's limits
    select_shape(S, species, shape);
    return EDUPIC_OK;
}

int edupic_get_push_shape(edupic_sim *S, int out[2])
{
    if (!S || !out) return EDUPIC_EINVAL;
    out[0] = S->shape[0];
    out[1] = S->shape[1];
    return EDUPIC_OK;
}

int edupic_describe_push_shape(int precision, int shape, int *threads, int *stages, int *min_blocks)
{
    if ((precision != EDUPIC_FP64 && precision != EDUPIC_FP32) || shape < 0 || shape >= kPushShapeCount)
        return EDUPIC_EINVAL;
    const PushShape p = push_shape_of(precision == EDUPIC_FP64, shape);
    if (threads) *threads = p.threads;
    if (stages) *stages = p.stages;
    if (min_blocks) *min_blocks = p.min_blocks;
    return EDUPIC_OK;
}

int edupic_autotune(edupic_sim *S, int subcycles, int measure, int out_blocks[2], double *out_ms_per_step)
{
    if (!S || subcycles < 1) return EDUPIC_EINVAL;
    if (!S->cs_set[0] || !S->cs_set[1]) return EDUPIC_ESTATE;
    if (S->phase != 0) return EDUPIC_ESTATE;  // trials are whole ion subcycles
    const int64_t steps = (int64_t)subcycles * S->nsub;
    int rc = EDUPIC_OK;
    // 1. launch shape of each species' particle kernel: every shape that fits
    // is timed on the live workload with an event pair around each launch
    // (both species in the same trial, each kernel on its own events); the
    // fastest mean launch per species is kept
    const int keep_shape[2] = {S->shape[0], S->shape[1]};
    int best_sh[2] = {keep_shape[0], keep_shape[1]};
    double best_t[2] = {-1.0, -1.0};
    for (int sh = 0; sh < kPushShapeCount && rc == EDUPIC_OK; ++sh) {
        bool fits[2];
        for (int sp = 0; sp < 2; ++sp) {
            fits[sp] = S->grid_shape[sp][sh] > 0;
            if (fits[sp]) select_shape(S, sp, sh);
        }
        if (!fits[0] && !fits[1]) continue;
        double ms[3];
        int64_t cnt[3];
        rc = edupic_profile_steps(S, S->nsub, measure, ms, cnt);  // warm
        if (rc == EDUPIC_OK) rc = edupic_profile_steps(S, steps, measure, ms, cnt);
        for (int sp = 0; sp < 2 && rc == EDUPIC_OK; ++sp) {
            if (!fits[sp] || cnt[sp] < 1) continue;
            const double t = ms[sp] / (double)cnt[sp];
            if (best_t[sp] < 0.0 || t < best_t[sp]) {
                best_t[sp] = t;
                best_sh[sp] = sh;
            }
        }
    }
    for (int sp = 0; sp < 2; ++sp) select_shape(S, sp, rc ? keep_shape[sp] : best_sh[sp]);
    if (rc) return rc;
    // 2. stepping mode: replay through one CUDA graph per ion subcycle, or
    // launch by launch (results are identical)
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return EDUPIC_ECUDA;
    const bool keep = S->graphs;
    bool best = keep;
    double best_ms = -1.0;
    for (int c = 0; c < 2 && rc == EDUPIC_OK; ++c) {
        const bool graphs = c == 0;
        S->graphs = graphs;
        if (!graphs) S->drop_graphs();
        rc = edupic_step(S, S->nsub, measure);  // warm (builds the graph when used)
        if (rc) break;
        cudaError_t e = cudaEventRecord(a, S->stream);
        if (e == cudaSuccess) rc = edupic_step(S, steps, measure);
        if (e == cudaSuccess && rc == EDUPIC_OK) e = cudaEventRecord(b, S->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) rc = EDUPIC_ECUDA;
        if (rc) break;
        if (best_ms < 0 || ms < best_ms) {
            best_ms = ms;
            best = graphs;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    S->graphs = rc ? keep : best;
    if (!S->graphs) S->drop_graphs();
    if (rc) return rc;
    if (out_blocks) {
        out_blocks[0] = S->grid[0];
        out_blocks[1] = S->grid[1];
    }
    if (out_ms_per_step) *out_ms_per_step = best_ms / (double)steps;
    return EDUPIC_OK;
}

int edupic_set_graphs(edupic_sim *S, int enable)
{
    if (!S) return EDUPIC_EINVAL;
    S->graphs = enable != 0;
    if (!S->graphs) S->drop_graphs();
    return EDUPIC_OK;
}

int edupic_get_graphs(edupic_sim *S, int *enabled)
{
    if (!S || !enabled) return EDUPIC_EINVAL;
    *enabled = S->graphs ? 1 : 0;
    return EDUPIC_OK;
}

int edupic_get_counts(edupic_sim *S, int d, int64_t *n_e, int64_t *n_i, int64_t *step)
{
    if (!valid_d(S, d)) return EDUPIC_EINVAL;
    Ctrl c;
    int rc = read_ctrl(S, d, &c);
    if (rc) return rc;
    if (n_e) *n_e = c.n[0];
    if (n_i) *n_i = c.n[1];
    if (step) *step = c.step;
    return error_of(c);
}

int edupic_get_particles(edupic_sim *S, int d, int species, int64_t cap, double *x, double *vx, double *vy,
                         double *vz, int64_t *n_out)
{
    if (!valid_d(S, d) || (species != 0 && species != 1) || cap < 0) return EDUPIC_EINVAL;
    Ctrl c;
    int rc = read_ctrl(S, d, &c);
    if (rc) return rc;
    const int64_t n = c.n[species];
    if (n_out) *n_out = n;
    const int64_t m = std::min<int64_t>(n, cap);
    double *dst[4] = {x, vx, vy, vz};
    rc = S->precision == EDUPIC_FP32 ? download_particles<float>(S, d, species, m, dst)
                                     : download_particles<double>(S, d, species, m, dst);
    if (rc) return rc;
    return error_of(c);
}

int edupic_get_fields(edupic_sim *S, int d, double *n_e, double *n_i, double *phi, double *efield, int64_t *q_e,
                      int64_t *q_i)
{
    if (!valid_d(S, d)) return EDUPIC_EINVAL;
    // densities and potential of the current step are formed on demand
    cudaError_t e0 = S->precision == EDUPIC_FP32 ? Launch<float>::fields(S->d_desc, S->nd, d, S->stream)
                                                 : Launch<double>::fields(S->d_desc, S->nd, d, S->stream);
    if (e0 != cudaSuccess || cudaStreamSynchronize(S->stream) != cudaSuccess) return EDUPIC_ECUDA;
    const DischargeDev &D = S->desc[d];
    const size_t ng = (size_t)S->params[d].n_grid;
    struct {
        void *dst;
        const void *src;
    } cp[6] = {{n_e, D.n_e}, {n_i, D.n_i}, {phi, D.phi}, {efield, D.ef}, {q_e, D.q_e}, {q_i, D.q_i}};
    for (auto &c : cp)
        if (c.dst && cudaMemcpy(c.dst, c.src, ng * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return EDUPIC_ECUDA;
    return EDUPIC_OK;
}

int edupic_get_diagnostics(edupic_sim *S, int d, double *ne_avg, double *ni_avg, double *phi_avg,
                           int64_t *eepf_counts, int64_t *ifed_pow_counts, int64_t *ifed_gnd_counts,
                           int64_t *measured_steps)
{
    if (!valid_d(S, d)) return EDUPIC_EINVAL;
    const DischargeDev &D = S->desc[d];
    const edupic_params &p = S->params[d];
    const size_t ng = (size_t)p.n_grid, ne = (size_t)kEepfStripes * p.eepf_bins, ni = (size_t)p.ifed_bins;
    // everything is queued into the page-locked stage behind the averages kernel; one synchronisation
    const size_t o_avg = align_up(sizeof(Ctrl), 16), o_eepf = o_avg + 3 * ng * 8, o_ifed = o_eepf + ne * 8;
    unsigned char *st = static_cast<unsigned char *>(pinned_reserve(S, o_ifed + 2 * ni * 8));
    if (!st) return EDUPIC_ENOMEM;
    double *outs[3] = {ne_avg, ni_avg, phi_avg};
    const bool avg = ne_avg || ni_avg || phi_avg;
    cudaError_t e = cudaMemcpyAsync(st, S->ctrl(d), sizeof(Ctrl), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess && avg) {
        e = S->precision == EDUPIC_FP32 ? Launch<float>::averages(S->d_desc, S->nd, d, S->stream)
                                        : Launch<double>::averages(S->d_desc, S->nd, d, S->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(st + o_avg, D.avg, 3 * ng * 8, cudaMemcpyDeviceToHost, S->stream);
    }
    if (e == cudaSuccess && eepf_counts)
        e = cudaMemcpyAsync(st + o_eepf, D.eepf, ne * 8, cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess && ifed_pow_counts)
        e = cudaMemcpyAsync(st + o_ifed, D.ifed_pow, ni * 8, cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess && ifed_gnd_counts)
        e = cudaMemcpyAsync(st + o_ifed + ni * 8, D.ifed_gnd, ni * 8, cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) return EDUPIC_ECUDA;
    Ctrl c;
    std::memcpy(&c, st, sizeof(Ctrl));
    const double *av = reinterpret_cast<const double *>(st + o_avg);
    for (int k = 0; k < 3; ++k)
        if (outs[k]) std::memcpy(outs[k], av + k * ng, ng * 8);
    if (eepf_counts) {
        const int64_t *h = reinterpret_cast<const int64_t *>(st + o_eepf);
        for (int b = 0; b < p.eepf_bins; ++b) {
            int64_t t = 0;
            for (int k = 0; k < kEepfStripes; ++k) t += h[(size_t)k * p.eepf_bins + b];
            eepf_counts[b] = t;
        }
    }
    if (ifed_pow_counts) std::memcpy(ifed_pow_counts, st + o_ifed, ni * 8);
    if (ifed_gnd_counts) std::memcpy(ifed_gnd_counts, st + o_ifed + ni * 8, ni * 8);
    if (measured_steps) *measured_steps = c.measured;
    return error_of(c);
}

int edupic_get_eepf(edupic_sim *S, int d, double *energy_ev, double *f)
{
    if (!valid_d(S, d)) return EDUPIC_EINVAL;
    const edupic_params &p = S->params[d];
    std::vector<int64_t> h((size_t)p.eepf_bins);
    int rc = edupic_get_diagnostics(S, d, nullptr, nullptr, nullptr, h.data(), nullptr, nullptr, nullptr);
    if (rc) return rc;
    double tot = 0.0;
    for (int64_t v : h) tot += (double)v;
    for (int k = 0; k < p.eepf_bins; ++k) {
        const double e = (k + 0.5) * p.eepf_de_ev;
        if (energy_ev) energy_ev[k] = e;
        if (f) f[k] = tot > 0 ? (double)h[k] / (tot * p.eepf_de_ev * std::sqrt(e)) : 0.0;
    }
    return EDUPIC_OK;
}

int edupic_get_ifed(edupic_sim *S, int d, double *energy_ev, double *f_pow, double *f_gnd)
{
    if (!valid_d(S, d)) return EDUPIC_EINVAL;
    const edupic_params &p = S->params[d];
    std::vector<int64_t> hp((size_t)p.ifed_bins), hg((size_t)p.ifed_bins);
    int rc = edupic_get_diagnostics(S, d, nullptr, nullptr, nullptr, nullptr, hp.data(), hg.data(), nullptr);
    if (rc) return rc;
    double tp = 0.0, tg = 0.0;
    for (int k = 0; k < p.ifed_bins; ++k) {
        tp += (double)hp[k];
        tg += (double)hg[k];
    }
    for (int k = 0; k < p.ifed_bins; ++k) {
        if (energy_ev) energy_ev[k] = (k + 0.5) * p.ifed_de_ev;
        if (f_pow) f_pow[k] = tp > 0 ? (double)hp[k] / (tp * p.ifed_de_ev) : 0.0;
        if (f_gnd) f_gnd[k] = tg > 0 ? (double)hg[k] / (tg * p.ifed_de_ev) : 0.0;
    }
    return EDUPIC_OK;
}

int edupic_get_counters(edupic_sim *S, int d, int64_t out[EDUPIC_N_COUNTERS])
{
    if (!valid_d(S, d) || !out) return EDUPIC_EINVAL;
    Ctrl c;
    int rc = read_ctrl(S, d, &c);
    if (rc) return rc;
    for (int k = 0; k < EDUPIC_N_COUNTERS; ++k) out[k] = (int64_t)c.counters[k];
    return error_of(c);
}

int edupic_reset_diagnostics(edupic_sim *S, int d)
{
    if (!valid_d(S, d)) return EDUPIC_EINVAL;
    const DischargeDev &D = S->desc[d];
    const edupic_params &p = S->params[d];
    const size_t ng = (size_t)p.n_grid;
    cudaError_t e = cudaMemsetAsync(D.sum_qe, 0, ng * 8, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.sum_qi, 0, ng * 8, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.sum_f, 0, ng * 8, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&D.fs->sum_V, 0, 2 * sizeof(double), S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.eepf, 0, (size_t)kEepfStripes * p.eepf_bins * 8, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.ifed_pow, 0, (size_t)p.ifed_bins * 8, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.ifed_gnd, 0, (size_t)p.ifed_bins * 8, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.power, 0, 2 * sizeof(double), S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&D.ctrl->measured, 0, sizeof(long long), S->stream);
    if (e == cudaSuccess && D.nxt > 0)
        e = cudaMemsetAsync(S->arena + S->base[d] + S->layouts[d].xt, 0, S->layouts[d].xt_bytes, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

// xt maps (Sec. 3.5) from the binned sums: the grid quantities through the
// same prefix-sum form as the time averages (per bin: sum phi_p = S_V + p S_d0
// - c sum_{j<p} S_F,j; E from the mean phi and the mean charge density at the
// edges), the particle quantities normalised per step of the bin.
int edupic_get_xt(edupic_sim *S, int d, int quantity, double *out)
{
    if (!valid_d(S, d) || !out || quantity < 0 || quantity >= EDUPIC_XT_QUANTITIES) return EDUPIC_EINVAL;
    const DischargeDev &D = S->desc[d];
    if (D.nxt < 1) return EDUPIC_ESTATE;
    Ctrl c;
    int rc = read_ctrl(S, d, &c);
    if (rc) return rc;
    const int ng = D.ng, nxt = D.nxt, M = ng - 1;
    const size_t m = (size_t)ng * nxt;
    std::vector<double> raw(9 * m + 2 * (size_t)nxt);
    std::vector<long long> steps(2 * (size_t)nxt);
    cudaError_t e = cudaMemcpy(raw.data(), D.xt_f, raw.size() * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(steps.data(), D.xt_steps, steps.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return EDUPIC_ECUDA;
    const double *F = raw.data(), *Qe = F + m, *Qi = F + 2 * m, *Ci = F + 3 * m, *Ve = F + 4 * m, *Vi = F + 5 * m;
    const double *Ee = F + 6 * m, *Ei = F + 7 * m, *Io = F + 8 * m, *SV = F + 9 * m, *Sd0 = SV + nxt;
    const double q2 = 1.0 / 4294967296.0;
    std::vector<double> phi((size_t)ng), ne((size_t)ng), ni((size_t)ng);
    for (int b = 0; b < nxt; ++b) {
        const double n0 = (double)steps[(size_t)b], n1 = (double)steps[(size_t)nxt + b];
        if (n0 <= 0.0) {
            for (int p = 0; p < ng; ++p) out[(size_t)p * nxt + b] = 0.0;
            continue;
        }
        double g = 0.0;
        for (int p = 0; p < ng; ++p) {
            const size_t j = (size_t)p * nxt + b;
            const double edge = (p == 0 || p == M) ? 2.0 : 1.0;
            phi[(size_t)p] = p == M ? 0.0 : (SV[b] + (double)p * Sd0[b] - D.poisson_c * g) / n0;
            if (p <= M - 1) g += F[j];
            ne[(size_t)p] = edge * D.factor_w * (Qe[j] * q2) / n0;
            ni[(size_t)p] = edge * D.factor_w * (Qi[j] * q2) / n0;
        }
        for (int p = 0; p < ng; ++p) {
            const size_t j = (size_t)p * nxt + b;
            const double edge = (p == 0 || p == M) ? 2.0 : 1.0;
            double ef;
            if (p == 0)
                ef = (phi[0] - phi[1]) / D.dx - kQE * (ni[0] - ne[0]) * D.dx / (2.0 * kEPS0);
            else if (p == M)
                ef = (phi[(size_t)M - 1] - phi[(size_t)M]) / D.dx + kQE * (ni[(size_t)M] - ne[(size_t)M]) * D.dx / (2.0 * kEPS0);
            else
                ef = (phi[(size_t)p - 1] - phi[(size_t)p + 1]) / (2.0 * D.dx);
            const double je = -kQE * D.factor_w * edge * Ve[j] / n0;
            const double ji = n1 > 0.0 ? kQE * D.factor_w * edge * Vi[j] / n1 : 0.0;
            double v = 0.0;
            switch (quantity) {
                case EDUPIC_XT_POT: v = phi[(size_t)p]; break;
                case EDUPIC_XT_EFIELD: v = ef; break;
                case EDUPIC_XT_NE: v = ne[(size_t)p]; break;
                case EDUPIC_XT_NI: v = ni[(size_t)p]; break;
                case EDUPIC_XT_JE: v = je; break;
                case EDUPIC_XT_JI: v = ji; break;
                case EDUPIC_XT_POWERE: v = je * ef; break;
                case EDUPIC_XT_POWERI: v = ji * ef; break;
                case EDUPIC_XT_MEANEE: v = Qe[j] > 0.0 ? Ee[j] / (Qe[j] * q2) : 0.0; break;
                case EDUPIC_XT_MEANEI: v = Ci[j] > 0.0 ? Ei[j] / (Ci[j] * q2) : 0.0; break;
                default: v = D.factor_w * edge * Io[j] / (n0 * D.dt_e); break;
            }
            out[j] = v;
        }
    }
    return error_of(c);
}

// Checkpoint file: magic, version, step, counts, then x, vx, vy, vz of the
// electrons and of the ions as FP64.
static const char kMagic[8] = {'E', 'D', 'U', 'P', 'I', 'C', 'C', 'K'};
static const int32_t kVersion = 1;

int edupic_save_state(edupic_sim *S, int d, const char *path)
{
    if (!valid_d(S, d) || !path) return EDUPIC_EINVAL;
    Ctrl c;
    int rc = read_ctrl(S, d, &c);
    if (rc) return rc;
    rc = error_of(c);
    if (rc) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return EDUPIC_EIO;
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
    const int32_t hdr[2] = {kVersion, S->params[d].n_grid};
    const int64_t vals[3] = {c.step, c.n[0], c.n[1]};
    ok = ok && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(vals, sizeof(vals), 1, f) == 1;
    for (int sp = 0; sp < 2 && ok; ++sp) {
        const int64_t n = c.n[sp];
        std::vector<double> a[4];
        double *dst[4];
        for (int k = 0; k < 4; ++k) {
            a[k].resize((size_t)n);
            dst[k] = a[k].data();
        }
        rc = S->precision == EDUPIC_FP32 ? download_particles<float>(S, d, sp, n, dst)
                                         : download_particles<double>(S, d, sp, n, dst);
        if (rc) {
            std::fclose(f);
            return rc;
        }
        for (int k = 0; k < 4 && ok; ++k) ok = std::fwrite(a[k].data(), 8, (size_t)n, f) == (size_t)n;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? EDUPIC_OK : EDUPIC_EIO;
}

int edupic_load_state(edupic_sim *S, int d, const char *path)
{
    if (!valid_d(S, d) || !path) return EDUPIC_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f) return EDUPIC_EIO;
    char magic[8];
    int32_t hdr[2];
    int64_t vals[3];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(vals, sizeof(vals), 1, f) == 1;
    ok = ok && hdr[0] == kVersion && hdr[1] == S->params[d].n_grid && vals[0] >= 0 && vals[1] >= 0 && vals[2] >= 0;
    if (!ok) {
        std::fclose(f);
        return EDUPIC_EIO;
    }
    if (vals[1] > S->params[d].capacity_e || vals[2] > S->params[d].capacity_i) {
        std::fclose(f);
        return EDUPIC_ECAPACITY;
    }
    // every discharge of an object steps on a common ion-subcycle phase
    if (vals[0] % S->nsub != S->phase) {
        std::fclose(f);
        return EDUPIC_ESTATE;
    }
    std::vector<double> a[2][4];
    for (int sp = 0; sp < 2 && ok; ++sp)
        for (int k = 0; k < 4 && ok; ++k) {
            a[sp][k].resize((size_t)vals[1 + sp]);
            ok = std::fread(a[sp][k].data(), 8, a[sp][k].size(), f) == a[sp][k].size();
        }
    ok = ok && std::fgetc(f) == EOF;  // a longer file is not a checkpoint of these counts
    std::fclose(f);
    if (!ok) return EDUPIC_EIO;
    // every value is checked before anything of the simulation changes
    for (int sp = 0; sp < 2; ++sp) {
        const double *src[4] = {a[sp][0].data(), a[sp][1].data(), a[sp][2].data(), a[sp][3].data()};
        if (!particles_valid(S, d, vals[1 + sp], src)) return EDUPIC_EINVAL;
    }
    long long step = vals[0];
    if (cudaMemcpy(&S->ctrl(d)->step, &step, sizeof(step), cudaMemcpyHostToDevice) != cudaSuccess)
        return EDUPIC_ECUDA;
    for (int sp = 0; sp < 2; ++sp) {
        int rc = edupic_load_particles(S, d, sp, vals[1 + sp], a[sp][0].data(), a[sp][1].data(), a[sp][2].data(),
                                       a[sp][3].data());
        if (rc) return rc;
    }
    return EDUPIC_OK;
}

int edupic_get_power(edupic_sim *S, int d, double out[2])
{
    if (!valid_d(S, d) || !out) return EDUPIC_EINVAL;
    Ctrl c;
    int rc = read_ctrl(S, d, &c);
    if (rc) return rc;
    double sums[2];
    if (cudaMemcpy(sums, S->desc[d].power, sizeof(sums), cudaMemcpyDeviceToHost) != cudaSuccess) return EDUPIC_ECUDA;
    const edupic_params &p = S->params[d];
    const DischargeDev &D = S->desc[d];
    // q E_x v_c dt summed per unit weight, with v_c = (v_old + v_new) / 2
    const double work[2] = {-kQE * 0.5 * sums[0] * D.dt_e, kQE * 0.5 * sums[1] * D.dt_i};
    const double t = (double)c.measured * D.dt_e;
    for (int k = 0; k < 2; ++k) out[k] = t > 0.0 ? work[k] * p.weight / (p.area_m2 * p.gap_m * t) : 0.0;
    return error_of(c);
}

int edupic_set_bias(edupic_sim *S, int d, double v_bias)
{
    if (!valid_d(S, d) || !std::isfinite(v_bias)) return EDUPIC_EINVAL;
    S->v_bias[(size_t)d] = v_bias;
    int rc = upload_drive(S, d);
    if (rc) return rc;
    // the field of the coming step was formed with the old drive: form it again
    cudaError_t e = S->precision == EDUPIC_FP32 ? Launch<float>::fields(S->d_desc, S->nd, d, S->stream)
                                                : Launch<double>::fields(S->d_desc, S->nd, d, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    return cuda_status(e);
}

int edupic_get_bias(edupic_sim *S, int d, double *v_bias)
{
    if (!valid_d(S, d) || !v_bias) return EDUPIC_EINVAL;
    *v_bias = S->v_bias[(size_t)d];
    return EDUPIC_OK;
}

int edupic_self_bias_step(edupic_sim *S, int64_t n_steps, int measure, const double *gain_v, double *v_bias)
{
    if (!S || n_steps < 1 || !gain_v) return EDUPIC_EINVAL;
    for (int d = 0; d < S->nd; ++d)
        if (!std::isfinite(gain_v[d])) return EDUPIC_EINVAL;
    std::vector<Ctrl> c0((size_t)S->nd), c1((size_t)S->nd);
    for (int d = 0; d < S->nd; ++d) {
        int rc = read_ctrl(S, d, &c0[(size_t)d]);
        if (rc) return rc;
    }
    int rc = edupic_step(S, n_steps, measure);
    if (rc == EDUPIC_OK) rc = edupic_synchronize(S);
    if (rc) return rc;
    for (int d = 0; d < S->nd; ++d) {
        rc = read_ctrl(S, d, &c1[(size_t)d]);
        if (rc) return rc;
        if (gain_v[d] != 0.0) {
            // charges reaching the powered electrode over the window: ions
            // (+), electrons (-), and the secondary electrons it emitted (+)
            const auto delta = [&](int k) { return (double)(c1[(size_t)d].counters[k] - c0[(size_t)d].counters[k]); };
            const double ni = delta(EDUPIC_C_ABS_I_POW), ne = delta(EDUPIC_C_ABS_E_POW), ns = delta(EDUPIC_C_EMITTED_POW);
            const double tot = ni + ne + ns;
            if (tot > 0.0) {
                rc = edupic_set_bias(S, d, S->v_bias[(size_t)d] + gain_v[d] * (ni - ne + ns) / tot);
                if (rc) return rc;
            }
        }
        if (v_bias) v_bias[d] = S->v_bias[(size_t)d];
    }
    return EDUPIC_OK;
}

int edupic_check_accuracy(edupic_sim *S, int d, edupic_accuracy *out)
{
    if (!valid_d(S, d) || !out) return EDUPIC_EINVAL;
    if (!S->cs_set[0] || !S->cs_set[1]) return EDUPIC_ESTATE;
    const edupic_params &p = S->params[d];
    const DischargeDev &D = S->desc[d];
    std::vector<double> ne((size_t)p.n_grid);
    std::vector<int64_t> h((size_t)p.eepf_bins);
    int64_t measured = 0;
    int rc = edupic_get_diagnostics(S, d, ne.data(), nullptr, nullptr, h.data(), nullptr, nullptr, &measured);
    if (rc) return rc;
    if (measured < 1) return EDUPIC_ESTATE;
    double nmax = 0.0;
    for (double v : ne) nmax = std::max(nmax, v);
    double cnt = 0.0, esum = 0.0;
    for (int k = 0; k < p.eepf_bins; ++k) {
        cnt += (double)h[k];
        esum += (double)h[k] * (k + 0.5) * p.eepf_de_ev;
    }
    edupic_accuracy a{};
    a.ne_max = nmax;
    a.te_ev = cnt > 0 ? (2.0 / 3.0) * esum / cnt : 0.0;  // effective temperature of the mean energy
    const double lambda_d = (nmax > 0 && a.te_ev > 0) ? std::sqrt(kEPS0 * a.te_ev * kQE / (nmax * kQE * kQE)) : 0.0;
    a.debye_ratio = lambda_d > 0 ? D.dx / lambda_d : 0.0;
    a.wpe_dt = std::sqrt(nmax * kQE * kQE / (kEPS0 * kME)) * D.dt_e;
    a.pcoll_max_e = 1.0 - std::exp(-D.n_gas * S->sigv_max[0] * D.dt_e);
    a.pcoll_max_i = 1.0 - std::exp(-D.n_gas * S->sigv_max[1] * D.dt_i);
    const double ve = D.dx / D.dt_e, vi = D.dx / D.dt_i;
    a.cfl_max_ev_e = 0.5 * kME * ve * ve / kQE;
    a.cfl_max_ev_i = 0.5 * (kArMassU * kAMU) * vi * vi / kQE;
    a.failed = (a.debye_ratio > 1.0 ? 1 : 0) | (a.wpe_dt >= 2.0 ? 2 : 0) |
               (a.pcoll_max_e >= 0.05 || a.pcoll_max_i >= 0.05 ? 4 : 0);
    *out = a;
    return a.failed ? EDUPIC_ESTABILITY : EDUPIC_OK;
}

const char *edupic_strerror(int status)
{
    switch (status) {
    case EDUPIC_OK: return "ok";
    case EDUPIC_EINVAL: return "invalid argument";
    case EDUPIC_ENOMEM: return "not enough device memory (arena or budget)";
    case EDUPIC_ECAPACITY: return "particle, hole or product capacity exceeded";
    case EDUPIC_ECUDA: return "CUDA runtime error";
    case EDUPIC_ESTATE: return "call not valid in the current state";
    case EDUPIC_ENAN: return "non-finite particle position";
    case EDUPIC_EIO: return "checkpoint file error";
    case EDUPIC_ETIMEOUT: return "bounded wait expired";
    case EDUPIC_ESTABILITY: return "an accuracy or stability condition fails (see edupic_check_accuracy)";
    case EDUPIC_ETOOBIG: return "n_grid exceeds the fixed scratch of the no-allocation entry point (max 2048)";
    default: return "unknown status";
    }
}

}  // extern "C"
