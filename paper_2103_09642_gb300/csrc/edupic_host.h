// Host-side state of a simulation object and the helpers shared by the C ABI
// translation units (edupic_api.cu: simulation objects; edupic_server.cu:
// the request server).  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "edupic_internal.h"

namespace edupic {
namespace host {

constexpr size_t kAlign = 256;    // alignment of every arena block
constexpr int kTileAlign = 1024;  // particle arrays padded to whole tiles

// Byte layout of one discharge inside the arena (offsets from its base).
struct Layout {
    size_t x[2], vx[2], vy[2], vz[2];
    size_t q_e, q_i, acc_e, acc_i, n_e, n_i, phi, ef, ef_t, f_cur, fs, sum_qe, sum_qi, sum_f, avg;
    size_t eepf, ifed_pow, ifed_gnd, power, holes[2], prod_parent, sort_buf, prod_x, prod_ve[3], prod_vi[3], vdrive;
    size_t emit_parent, emit_x, emit_v[3];  // present only when an electrode emits (see_gamma > 0)
    bool emit;
    size_t xt, xt_bytes;  // xt diagnostics block (xt_bins > 0), zeroed as one
    size_t sort_cnt, sort_tmp[4];  // periodic cell sort (sort_every > 0): chunk counts, scratch copy
    size_t bytes;
};

size_t align_up(size_t v, size_t a);
Layout layout_of(const edupic_params &p, size_t elem);
int check_params(int nd, const edupic_params *ps, int precision);
int cuda_status(cudaError_t e);

}  // namespace host
}  // namespace edupic

struct edupic_sim {
    int nd = 0, precision = 0;
    size_t elem = 8;
    std::vector<edupic_params> params;
    std::vector<edupic::host::Layout> layouts;
    std::vector<size_t> base;  // arena offset of each discharge
    std::vector<edupic::DischargeDev> desc;
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    edupic::DischargeDev *d_desc = nullptr;
    edupic::Ctrl *d_ctrl = nullptr;  // packed array: one per discharge
    void *cs_sig[2] = {nullptr, nullptr};
    void *cs_thr[2] = {nullptr, nullptr};
    void *cs_max[2] = {nullptr, nullptr};
    void *cs_pm[2] = {nullptr, nullptr};  // prefix maxima of sigma_tot * v per coarse block
    bool cs_set[2] = {false, false};
    cudaStream_t stream = nullptr;
    int ng_max = 0, eepf_max = 0, nsub = 1, nt_common = -1;
    int phase = 0;  // common step index modulo N_SUB
    int cs_shift_pending[2] = {0, 0};
    int lv_base_pending = 0, lv_n_pending = 1;  // e- bound table: first v^2 bucket, buckets
    int grid[2] = {0, 0};      // persistent grid of the particle kernel per species (its shape's resident limit)
    int grid_max[2] = {0, 0};  // resident limit (blocks per SM x SMs) of the shape in use
    int shape[2] = {0, 0};     // launch shape of the particle kernel per species (edupic_autotune)
    int grid_shape[2][edupic::kPushShapeCount] = {};  // resident limit of every shape (0: does not fit)
    int sms = 0;
    bool graphs = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double sigv_max[2] = {0.0, 0.0};  // largest sigma_tot * v of each species' table
    double sigv_top[2] = {0.0, 0.0};  // largest sigma_tot * v at the top of each entry's energy bin
    std::vector<double> sigsum_host[2];  // sum of the process cross sections per table entry (m^2)
    double cs_de_host[2] = {0.0, 0.0};
    int null_any[2] = {0, 0};  // some active discharge uses the null-collision method, per species
    int xt_any = 0;            // some discharge keeps xt diagnostics (the accumulating kernel variant)
    int sort_any = 0;          // some discharge sorts its particles by cell (sort_every > 0)
    int grid_xt[2] = {0, 0};   // resident limit of the accumulating particle kernel
    std::vector<double> v_bias;  // DC voltage added at the powered electrode, per discharge (Sec. 5 self-bias)
    void *pinned = nullptr;  // page-locked staging buffer for particle uploads
    size_t pinned_bytes = 0;

    ~edupic_sim()
    {
        for (auto &g : graph)
            if (g) cudaGraphExecDestroy(g);
        if (pinned) cudaFreeHost(pinned);
    }
    void drop_graphs()
    {
        for (auto &g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    edupic::Ctrl *ctrl(int d) const { return desc[d].ctrl; }
};

namespace edupic {
namespace host {

// bytes of the region shared by all discharges (descriptors, packed controls, tables)
size_t shared_bytes(int nd, size_t elem, int cs_entries);
// carve the shared region at the start of the arena
void carve_shared(edupic_sim *S, int cs_entries);
// persistent grid sizes of the particle kernels for the object's limits
int setup_grid(edupic_sim *S);
// fill the host copy of discharge d's descriptor from its params, layout and base
void fill_desc(edupic_sim *S, int d);
void null_bounds(edupic_sim *S, int d);
void update_null_any(edupic_sim *S);
int upload_desc(edupic_sim *S);
int upload_desc_one(edupic_sim *S, int d);
int upload_drive(edupic_sim *S, int d);
int load_species(edupic_sim *S, int d, int sp, int64_t n, const double *const src[4]);
cudaError_t enqueue_refresh(edupic_sim *S, int d, int sp);
int build_graph(edupic_sim *S, int measure);
int read_ctrl(edupic_sim *S, int d, Ctrl *c);
int error_of(const Ctrl &c);

}  // namespace host
}  // namespace edupic
