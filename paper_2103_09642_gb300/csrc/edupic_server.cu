// Request server of the C ABI (edupic_server_* in include/edupic.h):
// continuous batching of independent discharge simulations on one GPU.
//
// A server owns one simulation object with `max_slots` discharge slots.
// The particle and grid memory of a slot is carved on admission from a
// first-fit heap over the caller's arena (the HBM budget) and returned when
// the request finishes.  Every time step is one push launch per species and
// one finalize launch for all running slots, captured as one CUDA graph per
// ion subcycle.  Requests are admitted at ion-subcycle boundaries, so every
// slot's own step index keeps the common ion phase, and each slot stops at
// its own target step: the kernels skip a slot whose step count has reached
// its stop step, so a finished request is not advanced while the others run
// on.  A request's result therefore does not depend on what else ran beside
// it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "edupic_host.h"

using namespace edupic;
using namespace edupic::host;

namespace {

// First-fit allocator over [0, size) in kAlign units, with coalescing.
class Heap {
  public:
    explicit Heap(size_t size = 0) : size_(size)
    {
        if (size) free_[0] = size;
    }
    // returns the offset, or SIZE_MAX when no free block is large enough
    size_t alloc(size_t n)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            used_ += n;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n)
    {
        used_ -= std::min(used_, n);  // the block's own size, before it merges with free neighbours
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                n += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            free_.erase(next);
        }
        free_[off] = n;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

  private:
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    edupic_params p{};
    int64_t target = 0;       // time steps to run
    std::vector<double> part[2][4];
    int64_t n0[2] = {0, 0};
    int state = EDUPIC_REQ_QUEUED;
    int status = EDUPIC_OK;
    int slot = -1;
    size_t off = 0, bytes = 0;
    double t_submit = 0, t_admit = -1, t_done = -1;
    // results, read when the request finishes
    std::vector<double> avg;        // ne, ni, phi: 3 * n_grid
    std::vector<int64_t> eepf, ifed;  // eepf_bins; 2 * ifed_bins (powered, grounded)
    int64_t counters[EDUPIC_N_COUNTERS] = {};
    int64_t n_end[2] = {0, 0};
    int64_t steps_done = 0, measured = 0;
};

}  // namespace

struct edupic_server {
    edupic_sim *S = nullptr;
    edupic_server_config cfg{};
    size_t heap_base = 0;
    Heap heap;
    std::deque<uint64_t> queue;
    std::vector<uint64_t> slot_ticket;  // 0 = free slot
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    int64_t steps_run = 0;
    std::chrono::steady_clock::time_point t0;
    std::vector<Ctrl> ctrl_host;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    ~edupic_server() { delete S; }
};

namespace {

int check_config(const edupic_server_config *c)
{
    if (!c) return EDUPIC_EINVAL;
    if (c->max_slots < 1 || c->max_slots > EDUPIC_MAX_DISCHARGES) return EDUPIC_EINVAL;
    if (c->max_grid < 3 || c->max_grid > EDUPIC_MAX_GRID) return EDUPIC_EINVAL;
    if (c->max_eepf_bins < 1 || c->max_eepf_bins > EDUPIC_MAX_EEPF_BINS) return EDUPIC_EINVAL;
    if (c->ion_subcycle < 1 || c->cs_entries < 1) return EDUPIC_EINVAL;
    return EDUPIC_OK;
}

// Placeholder parameters of a free slot (never stepped: the slot is inactive).
edupic_params idle_params(const edupic_server_config &c)
{
    edupic_params p{};
    p.gap_m = 1.0;
    p.gas_temp_k = 300.0;
    p.area_m2 = 1.0;
    p.n_grid = 3;
    p.steps_per_cycle = c.ion_subcycle;
    p.ion_subcycle = c.ion_subcycle;
    p.cycle_freq_hz = 1.0;
    p.eepf_bins = 1;
    p.eepf_de_ev = 1.0;
    p.ifed_bins = 1;
    p.ifed_de_ev = 1.0;
    p.capacity_e = 1;
    p.capacity_i = 1;
    p.cs_entries = c.cs_entries;
    p.e_ion_ev = 1.0;
    return p;
}

DischargeDev idle_desc(edupic_sim *S, int d)
{
    DischargeDev D{};
    D.active = 0;
    D.stop_step = 0;
    D.ctrl = S->d_ctrl + d;
    for (int sp = 0; sp < 2; ++sp) {
        D.cs_sig[sp] = S->cs_sig[sp];
        D.cs_thr[sp] = S->cs_thr[sp];
        D.cs_max[sp] = S->cs_max[sp];
        D.cs_pm[sp] = S->cs_pm[sp];
    }
    // keep the table scalars set by edupic_server_set_cross_sections
    if ((size_t)d < S->desc.size()) {
        const DischargeDev &o = S->desc[d];
        D.cs_n_e = o.cs_n_e;
        D.cs_n_i = o.cs_n_i;
        D.cs_de_e = o.cs_de_e;
        D.cs_de_i = o.cs_de_i;
        D.inv_cs_de_ef = o.inv_cs_de_ef;
        D.inv_cs_de_if = o.inv_cs_de_if;
        D.e_idx_ef = o.e_idx_ef;
        D.g_idx_if = o.g_idx_if;
        D.cs_shift[0] = o.cs_shift[0];
        D.cs_shift[1] = o.cs_shift[1];
        D.lv_base = o.lv_base;
        D.lv_n = o.lv_n;
    }
    return D;
}

int check_request(const edupic_server *V, const edupic_params *p, int n_cycles)
{
    if (!p || n_cycles < 1) return EDUPIC_EINVAL;
    int rc = check_params(1, p, V->S->precision);
    if (rc) return rc;
    if (p->n_grid > V->cfg.max_grid || p->eepf_bins > V->cfg.max_eepf_bins) return EDUPIC_EINVAL;
    if (p->ion_subcycle != V->cfg.ion_subcycle || p->cs_entries != V->cfg.cs_entries) return EDUPIC_EINVAL;
    if (p->xt_bins != 0) return EDUPIC_EINVAL;  // xt maps are read from simulation objects only
    return EDUPIC_OK;
}

// Start request r in free slot d: carve its memory, fill and upload its
// descriptor, drive table and particles, and form the field of its step 0.
int open_slot(edupic_server *V, uint64_t ticket, int d)
{
    edupic_sim *S = V->S;
    Request &r = V->reqs[ticket];
    const size_t off = V->heap.alloc(r.bytes);
    if (off == SIZE_MAX) return EDUPIC_ENOMEM;
    r.off = off;
    S->params[d] = r.p;
    S->layouts[d] = layout_of(r.p, S->elem);
    S->base[d] = V->heap_base + off;
    cudaError_t e = cudaMemsetAsync(S->arena + S->base[d], 0, r.bytes, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->d_ctrl + d, 0, sizeof(Ctrl), S->stream);
    int rc = cuda_status(e);
    if (rc == EDUPIC_OK) {
        fill_desc(S, d);
        S->desc[d].stop_step = r.target;
        if (r.p.sort_every > 0 && !S->sort_any) {
            S->sort_any = 1;  // from now on every ion subcycle ends with the sort launches
            S->drop_graphs();
        }
        update_null_any(S);
        rc = upload_desc_one(S, d);
    }
    S->v_bias[(size_t)d] = 0.0;
    if (rc == EDUPIC_OK) rc = upload_drive(S, d);
    for (int sp = 0; sp < 2 && rc == EDUPIC_OK; ++sp) {
        const double *src[4] = {r.part[sp][0].data(), r.part[sp][1].data(), r.part[sp][2].data(),
                                r.part[sp][3].data()};
        rc = load_species(S, d, sp, r.n0[sp], src);
    }
    if (rc) {
        S->desc[d] = idle_desc(S, d);
        upload_desc_one(S, d);
        V->heap.release(off, r.bytes);
        return rc;
    }
    for (int sp = 0; sp < 2; ++sp)
        for (auto &a : r.part[sp]) std::vector<double>().swap(a);  // host copy no longer needed
    r.slot = d;
    r.state = EDUPIC_REQ_RUNNING;
    r.t_admit = V->now();
    V->slot_ticket[d] = ticket;
    return EDUPIC_OK;
}

// Return slot d and its heap memory (the slot's steps must have completed).
void free_slot(edupic_server *V, int d)
{
    edupic_sim *S = V->S;
    Request &r = V->reqs[V->slot_ticket[d]];
    S->desc[d] = idle_desc(S, d);
    update_null_any(S);
    upload_desc_one(S, d);
    V->heap.release(r.off, r.bytes);
    V->slot_ticket[d] = 0;
}

// Read the results of the request in slot d and free the slot.
void close_slot(edupic_server *V, int d, int status)
{
    edupic_sim *S = V->S;
    const uint64_t ticket = V->slot_ticket[d];
    Request &r = V->reqs[ticket];
    const edupic_params &p = r.p;
    r.avg.assign(3 * (size_t)p.n_grid, 0.0);
    r.eepf.assign((size_t)p.eepf_bins, 0);
    r.ifed.assign(2 * (size_t)p.ifed_bins, 0);
    int rc = status;
    if (rc == EDUPIC_OK) {
        const size_t ng = (size_t)p.n_grid;
        rc = edupic_get_diagnostics(S, d, r.avg.data(), r.avg.data() + ng, r.avg.data() + 2 * ng, r.eepf.data(),
                                    r.ifed.data(), r.ifed.data() + p.ifed_bins, &r.measured);
    }
    Ctrl c{};
    if (read_ctrl(S, d, &c) == EDUPIC_OK) {
        for (int k = 0; k < EDUPIC_N_COUNTERS; ++k) r.counters[k] = (int64_t)c.counters[k];
        r.n_end[0] = c.n[0];
        r.n_end[1] = c.n[1];
        r.steps_done = c.step;
    }
    r.status = rc;
    r.state = rc == EDUPIC_OK ? EDUPIC_REQ_DONE : EDUPIC_REQ_FAILED;
    r.t_done = V->now();
    free_slot(V, d);
}

}  // namespace

extern "C" {

int edupic_server_arena_bytes(const edupic_server_config *cfg, int precision, size_t heap_bytes, size_t *bytes)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!bytes || (precision != EDUPIC_FP64 && precision != EDUPIC_FP32)) return EDUPIC_EINVAL;
    const size_t elem = precision == EDUPIC_FP32 ? 4 : 8;
    *bytes = align_up(shared_bytes(cfg->max_slots, elem, cfg->cs_entries), kAlign) + align_up(heap_bytes, kAlign);
    return EDUPIC_OK;
}

int edupic_server_create(const edupic_server_config *cfg, int precision, void *device_arena, size_t arena_bytes,
                         void *cuda_stream, edupic_server **out)
{
    if (!out) return EDUPIC_EINVAL;
    *out = nullptr;
    size_t need = 0;
    int rc = edupic_server_arena_bytes(cfg, precision, 0, &need);
    if (rc) return rc;
    if (!device_arena || ((uintptr_t)device_arena % kAlign)) return EDUPIC_EINVAL;
    if (arena_bytes < need) return EDUPIC_ENOMEM;
    edupic_server *V = new (std::nothrow) edupic_server();
    if (!V) return EDUPIC_ENOMEM;
    V->cfg = *cfg;
    V->t0 = std::chrono::steady_clock::now();
    edupic_sim *S = new (std::nothrow) edupic_sim();
    if (!S) {
        delete V;
        return EDUPIC_ENOMEM;
    }
    V->S = S;
    const int nd = cfg->max_slots;
    S->nd = nd;
    S->precision = precision;
    S->elem = precision == EDUPIC_FP32 ? 4 : 8;
    S->arena = static_cast<unsigned char *>(device_arena);
    S->arena_bytes = arena_bytes;
    S->stream = static_cast<cudaStream_t>(cuda_stream);
    S->nsub = cfg->ion_subcycle;
    S->nt_common = -1;
    S->ng_max = cfg->max_grid;
    S->eepf_max = cfg->max_eepf_bins;
    carve_shared(S, cfg->cs_entries);
    S->params.assign(nd, idle_params(*cfg));
    S->v_bias.assign((size_t)nd, 0.0);
    S->layouts.assign(nd, Layout{});
    S->base.assign(nd, 0);
    S->desc.clear();
    for (int d = 0; d < nd; ++d) S->desc.push_back(idle_desc(S, d));
    V->heap_base = need;
    V->heap = Heap((arena_bytes - need) / kAlign * kAlign);
    V->slot_ticket.assign(nd, 0);
    V->ctrl_host.resize(nd);
    cudaError_t e = cudaMemsetAsync(S->arena, 0, need, S->stream);
    rc = cuda_status(e);
    if (rc == EDUPIC_OK) rc = upload_desc(S);
    if (rc == EDUPIC_OK) rc = setup_grid(S);
    if (rc) {
        delete V;
        return rc;
    }
    *out = V;
    return EDUPIC_OK;
}

int edupic_server_destroy(edupic_server *V)
{
    if (!V) return EDUPIC_EINVAL;
    if (V->S && V->S->stream) cudaStreamSynchronize(V->S->stream);
    delete V;
    return EDUPIC_OK;
}

int edupic_server_set_cross_sections(edupic_server *V, int species, int n_proc, int n_entries, double de_ev,
                                     const double *sigma_m2)
{
    if (!V) return EDUPIC_EINVAL;
    for (uint64_t t : V->slot_ticket)
        if (t) return EDUPIC_ESTATE;  // tables are shared by every running request
    return edupic_set_cross_sections(V->S, species, n_proc, n_entries, de_ev, sigma_m2);
}

int edupic_server_request_bytes(const edupic_server *V, const edupic_params *p, size_t *bytes)
{
    if (!V || !bytes) return EDUPIC_EINVAL;
    int rc = check_request(V, p, 1);
    if (rc) return rc;
    *bytes = layout_of(*p, V->S->elem).bytes;
    return EDUPIC_OK;
}

int edupic_server_submit(edupic_server *V, const edupic_params *p, int n_cycles, int64_t n_e,
                         const double *const e[4], int64_t n_i, const double *const i[4], uint64_t *ticket)
{
    if (!V || !ticket) return EDUPIC_EINVAL;
    int rc = check_request(V, p, n_cycles);
    if (rc) return rc;
    const int64_t n[2] = {n_e, n_i};
    const double *const *src[2] = {e, i};
    for (int sp = 0; sp < 2; ++sp) {
        if (n[sp] < 0) return EDUPIC_EINVAL;
        if (n[sp] > (sp == 0 ? p->capacity_e : p->capacity_i)) return EDUPIC_ECAPACITY;
        if (n[sp] > 0 && (!src[sp] || !src[sp][0] || !src[sp][1] || !src[sp][2] || !src[sp][3])) return EDUPIC_EINVAL;
        for (int64_t j = 0; j < n[sp]; ++j)
            if (!(src[sp][0][j] >= 0.0 && src[sp][0][j] <= p->gap_m) || !std::isfinite(src[sp][1][j]) ||
                !std::isfinite(src[sp][2][j]) || !std::isfinite(src[sp][3][j]))
                return EDUPIC_EINVAL;
    }
    const size_t bytes = layout_of(*p, V->S->elem).bytes;
    if (bytes > V->heap.size()) return EDUPIC_ENOMEM;  // can never fit the budget
    Request r;
    r.p = *p;
    r.target = (int64_t)n_cycles * p->steps_per_cycle;
    r.bytes = bytes;
    for (int sp = 0; sp < 2; ++sp) {
        r.n0[sp] = n[sp];
        for (int c = 0; c < 4; ++c) r.part[sp][c].assign(src[sp] ? src[sp][c] : nullptr,
                                                         src[sp] ? src[sp][c] + n[sp] : nullptr);
    }
    r.t_submit = V->now();
    const uint64_t t = V->next_ticket++;
    V->reqs.emplace(t, std::move(r));
    V->queue.push_back(t);
    *ticket = t;
    return EDUPIC_OK;
}

int edupic_server_advance(edupic_server *V, int n_subcycles, int *n_running, int *n_queued)
{
    if (!V || n_subcycles < 0) return EDUPIC_EINVAL;
    edupic_sim *S = V->S;
    if (!S->cs_set[0] || !S->cs_set[1]) return EDUPIC_ESTATE;
    // 1. wait for the steps enqueued last time and retire finished requests
    if (cudaStreamSynchronize(S->stream) != cudaSuccess) return EDUPIC_ECUDA;
    if (cudaMemcpy(V->ctrl_host.data(), S->d_ctrl, sizeof(Ctrl) * S->nd, cudaMemcpyDeviceToHost) != cudaSuccess)
        return EDUPIC_ECUDA;
    for (int d = 0; d < S->nd; ++d) {
        if (!V->slot_ticket[d]) continue;
        const Ctrl &c = V->ctrl_host[d];
        const Request &r = V->reqs[V->slot_ticket[d]];
        if (c.error) close_slot(V, d, error_of(c));
        else if (c.step >= r.target) close_slot(V, d, EDUPIC_OK);
    }
    // 2. admit queued requests in arrival order while a slot and memory are free
    while (!V->queue.empty()) {
        int d = 0;
        while (d < S->nd && V->slot_ticket[d]) ++d;
        if (d == S->nd) break;
        const uint64_t t = V->queue.front();
        int rc = open_slot(V, t, d);
        if (rc == EDUPIC_ENOMEM) break;  // wait until running requests free memory
        V->queue.pop_front();
        if (rc) {
            Request &r = V->reqs[t];
            r.state = EDUPIC_REQ_FAILED;
            r.status = rc;
            r.t_done = V->now();
        }
    }
    // 3. enqueue the next ion subcycles for every running slot
    int running = 0;
    for (uint64_t t : V->slot_ticket) running += t ? 1 : 0;
    if (running && n_subcycles) {
        int rc = edupic_step(S, (int64_t)n_subcycles * S->nsub, 1);
        if (rc) return rc;
        V->steps_run += (int64_t)n_subcycles * S->nsub;
    }
    if (n_running) *n_running = running;
    if (n_queued) *n_queued = (int)V->queue.size();
    return EDUPIC_OK;
}

int edupic_server_info(edupic_server *V, uint64_t ticket, edupic_request_info *info)
{
    if (!V || !info) return EDUPIC_EINVAL;
    auto it = V->reqs.find(ticket);
    if (it == V->reqs.end()) return EDUPIC_EINVAL;
    const Request &r = it->second;
    info->state = r.state;
    info->status = r.status;
    info->slot = r.slot;
    info->reserved = 0;
    info->steps_target = r.target;
    info->steps_done = r.steps_done;
    info->n_e = r.state == EDUPIC_REQ_QUEUED || r.state == EDUPIC_REQ_RUNNING ? r.n0[0] : r.n_end[0];
    info->n_i = r.state == EDUPIC_REQ_QUEUED || r.state == EDUPIC_REQ_RUNNING ? r.n0[1] : r.n_end[1];
    info->bytes = (int64_t)r.bytes;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    return EDUPIC_OK;
}

int edupic_server_result(edupic_server *V, uint64_t ticket, double *ne_avg, double *ni_avg, double *phi_avg,
                         int64_t *eepf_counts, int64_t *ifed_pow_counts, int64_t *ifed_gnd_counts,
                         int64_t counters[EDUPIC_N_COUNTERS], int64_t *measured_steps)
{
    if (!V) return EDUPIC_EINVAL;
    auto it = V->reqs.find(ticket);
    if (it == V->reqs.end()) return EDUPIC_EINVAL;
    const Request &r = it->second;
    if (r.state == EDUPIC_REQ_FAILED) return r.status ? r.status : EDUPIC_ESTATE;
    if (r.state != EDUPIC_REQ_DONE) return EDUPIC_ESTATE;
    const size_t ng = (size_t)r.p.n_grid, nb = (size_t)r.p.ifed_bins;
    if (ne_avg) std::copy(r.avg.begin(), r.avg.begin() + ng, ne_avg);
    if (ni_avg) std::copy(r.avg.begin() + ng, r.avg.begin() + 2 * ng, ni_avg);
    if (phi_avg) std::copy(r.avg.begin() + 2 * ng, r.avg.end(), phi_avg);
    if (eepf_counts) std::copy(r.eepf.begin(), r.eepf.end(), eepf_counts);
    if (ifed_pow_counts) std::copy(r.ifed.begin(), r.ifed.begin() + nb, ifed_pow_counts);
    if (ifed_gnd_counts) std::copy(r.ifed.begin() + nb, r.ifed.end(), ifed_gnd_counts);
    if (counters) std::copy(r.counters, r.counters + EDUPIC_N_COUNTERS, counters);
    if (measured_steps) *measured_steps = r.measured;
    return EDUPIC_OK;
}

int edupic_server_release(edupic_server *V, uint64_t ticket)
{
    if (!V) return EDUPIC_EINVAL;
    auto it = V->reqs.find(ticket);
    if (it == V->reqs.end()) return EDUPIC_EINVAL;
    Request &r = it->second;
    if (r.state == EDUPIC_REQ_QUEUED) {
        V->queue.erase(std::find(V->queue.begin(), V->queue.end(), ticket));
    } else if (r.state == EDUPIC_REQ_RUNNING) {
        // cancelled mid-run: the steps already enqueued complete first, then
        // the slot and its memory are returned; other slots are not touched
        if (cudaStreamSynchronize(V->S->stream) != cudaSuccess) return EDUPIC_ECUDA;
        free_slot(V, r.slot);
    }
    V->reqs.erase(it);
    return EDUPIC_OK;
}

int edupic_server_stats(edupic_server *V, edupic_server_stats_t *out)
{
    if (!V || !out) return EDUPIC_EINVAL;
    out->now = V->now();
    out->steps_run = V->steps_run;
    out->heap_bytes = (int64_t)V->heap.size();
    out->heap_used = (int64_t)V->heap.used();
    int running = 0;
    for (uint64_t t : V->slot_ticket) running += t ? 1 : 0;
    out->running = running;
    out->queued = (int)V->queue.size();
    return EDUPIC_OK;
}

}  // extern "C"
