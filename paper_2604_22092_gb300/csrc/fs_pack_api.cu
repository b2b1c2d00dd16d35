// fs_pack_api.cu -- C ABI of packed ensembles and batches (include/fs.h):
// ensemble state node-major on the device, and the batch's segment table,
// stepped by one launch per step (replays of a captured graph; members join
// and leave between launches, the table is re-uploaded only then).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fs.h"
#include "fs_launch.h"
#include "fs_objects.h"

using fsapi::dev_alloc;
using fsapi::fail;
using fsapi::g_err;

struct fs_batch;

struct fs_ens {
    fs_graph* g = nullptr;
    int32_t R = 0, R_pad = 8, age_dtype = 0, model = 0;
    int age_bytes = 4, mask_bytes = 1;
    uint8_t* d_X = nullptr;
    void* d_A = nullptr;
    void* d_mask[2] = {nullptr, nullptr};
    // push form of the pressure (push = true): counts and pending tallies
    bool push = false;
    uint8_t* d_pc8 = nullptr;
    uint16_t* d_ppd[2] = {nullptr, nullptr};
    uint32_t* d_phc = nullptr;
    unsigned long long* d_phpd[2] = {nullptr, nullptr};
    fs::PackScen* d_scen = nullptr;
    // adaptive step (every realisation has eps > 0): the rate ring and the
    // per-replicate clocks
    uint32_t* d_lam = nullptr;
    double* d_time = nullptr;
    // shedding profile (every realisation has one, gather form): the
    // infectivity of each (node, replicate) by local step parity and each
    // scenario's memoised beta s(age) table
    bool shed = false;
    void* d_rho[2] = {nullptr, nullptr};
    float4* d_rtab = nullptr;
    std::vector<fs::PackScen> h_scen;
    float4* d_ptab = nullptr;
    float* d_ps = nullptr;
    unsigned long long* d_deltas = nullptr;
    uint32_t* d_counts = nullptr;
    uint32_t* d_out = nullptr;          // counts rows of the current membership
    int64_t steps_done = 0;             // the ensemble's step index
    fs_batch* batch = nullptr;          // live membership
    cudaStream_t stream = nullptr;
    int64_t bytes = 0;
    bool failed = false;
};

namespace {

struct Member {
    fs_ens* e;
    int64_t g_join;          // global step of the member's first launch
    int64_t steps;
    uint32_t* host_out;
};

}  // namespace

struct fs_batch {
    int32_t age_dtype = 0;
    int32_t cap = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    fs::PackSeg* d_seg = nullptr;
    int64_t* d_thr = nullptr;
    int64_t* d_hub = nullptr;
    int32_t* d_cls = nullptr;           // [kPackClasses + 1] class boundaries of the table (see PackArgs)
    fs::PackSeg* h_seg = nullptr;       // pinned staging of the table
    int64_t* h_thr = nullptr;
    int64_t* h_hub = nullptr;
    int32_t* h_cls = nullptr;
    fs::DevCtl* d_ctl = nullptr;
    int64_t G = 0;                      // global step of the next launch
    std::vector<Member> members;
    bool dirty = true;
    cudaGraphExec_t gexec = nullptr;
    int gK = 0;
    int g_classes = 0;                  // classes launched by the captured graph (bit c)
    int classes = 0;                    // classes present in the table (bit (3c+f)*2+d: R_pad = 8 << c, form f
                                        // (0 gather, 1 push, 2 gather with shedding), step d = adaptive)
    int grid[3] = {0, 0, 0};
    bool failed = false;
};

namespace {

void free_ens(fs_ens* e)
{
    if (!e)
        return;
    fs::dfree(e->d_X);
    fs::dfree(e->d_A);
    fs::dfree(e->d_mask[0]);
    fs::dfree(e->d_mask[1]);
    fs::dfree(e->d_pc8);
    fs::dfree(e->d_ppd[0]);
    fs::dfree(e->d_ppd[1]);
    fs::dfree(e->d_phc);
    fs::dfree(e->d_phpd[0]);
    fs::dfree(e->d_phpd[1]);
    fs::dfree(e->d_scen);
    fs::dfree(e->d_ptab);
    fs::dfree(e->d_ps);
    fs::dfree(e->d_deltas);
    fs::dfree(e->d_counts);
    fs::dfree(e->d_out);
    fs::dfree(e->d_lam);
    fs::dfree(e->d_time);
    fs::dfree(e->d_rho[0]);
    fs::dfree(e->d_rho[1]);
    fs::dfree(e->d_rtab);
    if (e->stream)
        cudaStreamDestroy(e->stream);
    delete e;
}

void free_batch(fs_batch* b)
{
    if (!b)
        return;
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    fs::dfree(b->d_seg);
    fs::dfree(b->d_thr);
    fs::dfree(b->d_hub);
    fs::dfree(b->d_cls);
    fs::dfree(b->d_ctl);
    cudaFreeHost(b->h_seg);
    cudaFreeHost(b->h_thr);
    cudaFreeHost(b->h_hub);
    cudaFreeHost(b->h_cls);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
}

fs::PackSeg segment_of(const Member& m)
{
    const fs_ens* e = m.e;
    const fs_graph* g = e->g;
    fs::PackSeg s{};
    s.sell_off = g->d_sell_off;
    s.sell_col = g->d_sell_col;
    s.m_ptr = g->d_m_ptr;
    s.m_col = g->d_m_col;
    s.perm = g->d_perm;
    s.n = (int32_t)g->n;
    s.n_thr = g->n_thr;
    s.n_slices = g->n_slices;
    s.n_m = g->n_m;
    s.sentinel = (int32_t)g->n;
    s.R_pad = e->R_pad;
    s.R = e->R;
    s.model = e->model;
    s.X = e->d_X;
    s.A = e->d_A;
    s.mask[0] = e->d_mask[0];
    s.mask[1] = e->d_mask[1];
    s.scen = e->d_scen;
    s.kmin = e->steps_done;
    s.kend = e->steps_done + m.steps;
    s.join = m.g_join - e->steps_done;
    s.deltas = e->d_deltas;
    s.counts = e->d_counts;
    s.out = e->d_out;
    s.push = e->push ? 1 : 0;
    s.pc8 = e->d_pc8;
    s.ppd[0] = e->d_ppd[0];
    s.ppd[1] = e->d_ppd[1];
    s.phc = e->d_phc;
    s.phpd[0] = e->d_phpd[0];
    s.phpd[1] = e->d_phpd[1];
    s.out_ptr = g->d_out_ptr;
    s.out_col = g->d_out_col;
    s.lam = e->d_lam;
    s.time = e->d_time;
    s.shed = e->shed ? 1 : 0;
    s.rho[0] = e->d_rho[0];
    s.rho[1] = e->d_rho[1];
    return s;
}

}  // namespace

namespace fsapi {

// FS_PRESSURE_AUTO for a packed ensemble: the push form at 8 replicate lanes,
// the gather at 16 and 32, where a gather's column and mask reads serve more
// replicates than its pushes cost (measured on GB300, 400-step SEIR runs,
// packed gather / push GNUPS: ER d = 8, N = 10^6: 119 / 156 at 8 lanes,
// 148 / 127 at 16, 151 / 136 at 32; BA m = 4: 108 / 113, 119 / 103,
// 119 / 108; regular d = 10, N = 3 x 10^5: 85 / 107, 108 / 118, 116 / 111).
// A shedding profile needs the gather.
bool packed_push(const fs_graph* g, const fs_sim_params& p0, int n_real)
{
    if (p0.flags == FS_PRESSURE_PUSH)
        return true;
    return p0.flags == FS_PRESSURE_AUTO && p0.shed_mode == FS_SHED_NONE && n_real <= 8 && push_available(g);
}

}  // namespace fsapi

#define E_CUDA(obj, expr)                                                                                    \
    do {                                                                                                     \
        cudaError_t e_ = (expr);                                                                             \
        if (e_ != cudaSuccess) {                                                                             \
            (obj)->failed = true;                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA, "%s: %s", #expr,           \
                        cudaGetErrorString(e_));                                                             \
        }                                                                                                    \
    } while (0)

extern "C" {

fs_status fs_ens_create(fs_graph* g, const fs_sim_params* params, int32_t n_real, const int32_t* index_nodes,
                        int64_t n_index, fs_ens** out)
{
    g_err.clear();
    if (!g || !params || !out)
        return fail(FS_EINVAL, "fs_ens_create: NULL argument");
    *out = nullptr;
    if (g->failed)
        return fail(FS_ESTATE, "fs_ens_create: graph is in a failed state");
    if (n_real < 1 || n_real > fs::kPackMaxR)
        return fail(FS_EINVAL, "fs_ens_create: n_real must be in [1, %d]", fs::kPackMaxR);
    for (int r = 0; r < n_real; ++r) {
        fs_status st = fsapi::check_params(params + r);
        if (st != FS_OK)
            return st;
        if (params[r].model != params[0].model || params[r].age_dtype != params[0].age_dtype ||
            params[r].index_state != params[0].index_state || params[r].flags != params[0].flags)
            return fail(FS_EINVAL, "fs_ens_create: realisations must share model, age_dtype, index_state and flags");
    }
    for (int r = 0; r < n_real; ++r) {
        if ((params[r].eps > 0) != (params[0].eps > 0))
            return fail(FS_EINVAL, "fs_ens_create: every realisation takes the adaptive step (eps > 0) or none");
        if ((params[r].shed_mode != FS_SHED_NONE) != (params[0].shed_mode != FS_SHED_NONE))
            return fail(FS_EINVAL, "fs_ens_create: every realisation has a shedding profile or none");
        if (params[r].flags & FS_ACTIVE_LIST)
            return fail(FS_EUNSUPPORTED, "fs_ens_create: FS_ACTIVE_LIST is for single realisations");
        if (params[r].theta > 0)
            return fail(FS_EUNSUPPORTED, "fs_ens_create: the Markovian engine is for single realisations");
    }
    if (params[0].shed_mode != FS_SHED_NONE && params[0].flags == FS_PRESSURE_PUSH)
        return fail(FS_EUNSUPPORTED, "fs_ens_create: a shedding profile needs the gather form of the pressure");
    if (params[0].flags == FS_PRESSURE_PUSH && !fsapi::push_available(g))
        return fail(FS_EUNSUPPORTED, "fs_ens_create: FS_PRESSURE_PUSH needs in-degrees <= %d in the thread class",
                    fs::kMaxThreadDeg);
    if (n_index < 0 || n_index > g->n || (n_index > 0 && !index_nodes))
        return fail(FS_EINVAL, "fs_ens_create: bad index list size");
    {
        std::vector<int32_t> v(index_nodes, index_nodes + n_index);
        std::sort(v.begin(), v.end());
        for (int64_t q = 0; q < n_index; ++q) {
            if (v[q] < 0 || v[q] >= g->n)
                return fail(FS_EINVAL, "fs_ens_create: index node %d out of range", v[q]);
            if (q && v[q] == v[q - 1])
                return fail(FS_EINVAL, "fs_ens_create: index node %d repeated", v[q]);
        }
    }
    fs_ens* e = new fs_ens();
    e->g = g;
    e->R = n_real;
    e->R_pad = n_real <= 8 ? 8 : n_real <= 16 ? 16 : 32;
    e->age_dtype = params[0].age_dtype;
    e->model = params[0].model;
    e->age_bytes = e->age_dtype == FS_AGE_F32 ? 4 : 2;
    e->mask_bytes = e->R_pad / 8;
    e->push = fsapi::packed_push(g, params[0], n_real);
    e->shed = params[0].shed_mode != FS_SHED_NONE;
    const int64_t n = g->n;
    const int Rp = e->R_pad;
    int32_t* d_idx = nullptr;
    auto bail = [&](fs_status st) {
        fs::dfree(d_idx);
        free_ens(e);
        return st;
    };
#define C_TRY(expr)                                                                                          \
    do {                                                                                                     \
        cudaError_t e_ = (expr);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA, "%s: %s", #expr,      \
                             cudaGetErrorString(e_)));                                                       \
    } while (0)
    C_TRY(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
    cudaStream_t cs = e->stream;
    C_TRY(dev_alloc(&e->d_X, (size_t)n * Rp, &e->bytes));
    C_TRY(fs::dmalloc(&e->d_A, (size_t)n * Rp * e->age_bytes));
    e->bytes += (int64_t)n * Rp * e->age_bytes;
    for (int q = 0; q < 2; ++q) {
        C_TRY(fs::dmalloc(&e->d_mask[q], (size_t)(n + 1) * e->mask_bytes));
        e->bytes += (int64_t)(n + 1) * e->mask_bytes;
        C_TRY(cudaMemsetAsync(e->d_mask[q], 0, (size_t)(n + 1) * e->mask_bytes, cs));
    }
    C_TRY(dev_alloc(&e->d_scen, (size_t)Rp, &e->bytes));
    C_TRY(dev_alloc(&e->d_ptab, (size_t)n_real * 2 * fs::kPTableN, &e->bytes));
    C_TRY(dev_alloc(&e->d_ps, (size_t)n_real * fs::kPSTableN, &e->bytes));
    C_TRY(dev_alloc(&e->d_deltas, (size_t)2 * Rp * 3, &e->bytes));
    C_TRY(dev_alloc(&e->d_counts, (size_t)Rp * 4, &e->bytes));
    C_TRY(cudaMemsetAsync(e->d_A, 0, (size_t)n * Rp * e->age_bytes, cs));
    C_TRY(cudaMemsetAsync(e->d_deltas, 0, sizeof(unsigned long long) * 2 * Rp * 3, cs));
    C_TRY(cudaMemsetAsync(e->d_ptab, 0xff, sizeof(float4) * n_real * 2 * fs::kPTableN, cs));
    if (e->shed) {
        for (int q = 0; q < 2; ++q) {
            C_TRY(fs::dmalloc(&e->d_rho[q], (size_t)n * Rp * e->age_bytes));
            e->bytes += (int64_t)n * Rp * e->age_bytes;
        }
        C_TRY(dev_alloc(&e->d_rtab, (size_t)n_real * fs::kPTableN, &e->bytes));
        C_TRY(cudaMemsetAsync(e->d_rtab, 0xff, sizeof(float4) * n_real * fs::kPTableN, cs));
    }
    std::vector<fs::PackScen> scen(Rp);
    for (int r = 0; r < n_real; ++r) {
        fs::PackScen sc{};
        sc.M = fsapi::to_model(params[r]);
        sc.ptab = e->d_ptab + (size_t)r * 2 * fs::kPTableN;
        sc.ps = e->d_ps + (size_t)r * fs::kPSTableN;
        sc.key0 = sc.M.key0;
        sc.key1 = sc.M.key1;
        sc.rep = sc.M.rep;
        sc.dt = sc.M.dt;
        sc.beta = sc.M.beta;
        sc.inv_dt = sc.M.inv_dt;
        sc.eps = (float)params[r].eps;
        sc.delta = (float)(params[r].delta > 0 ? params[r].delta : 1e-12);
        if (e->shed) {
            sc.rtab = e->d_rtab + (size_t)r * fs::kPTableN;
            sc.shed = fsapi::to_lawf(params[r].shedding);
            sc.shed_mode = params[r].shed_mode;
        }
        C_TRY(fs::launch_build_ptables(sc.M, e->age_dtype, const_cast<float4*>(sc.ptab), const_cast<float*>(sc.ps),
                                       cs, const_cast<float4*>(sc.rtab), sc.shed, sc.shed_mode));
        scen[r] = sc;
    }
    for (int r = n_real; r < Rp; ++r)
        scen[r] = scen[0];                       // padding replicates never draw
    C_TRY(cudaMemcpyAsync(e->d_scen, scen.data(), sizeof(fs::PackScen) * Rp, cudaMemcpyHostToDevice, cs));
    e->h_scen = scen;
    if (params[0].eps > 0) {
        C_TRY(dev_alloc(&e->d_lam, (size_t)3 * Rp, &e->bytes));
        C_TRY(dev_alloc(&e->d_time, (size_t)Rp, &e->bytes));
        C_TRY(cudaMemsetAsync(e->d_lam, 0, sizeof(uint32_t) * 3 * Rp, cs));
        C_TRY(cudaMemsetAsync(e->d_time, 0, sizeof(double) * Rp, cs));
    }
    if (n_index > 0) {
        C_TRY(dev_alloc(&d_idx, (size_t)n_index, nullptr));
        C_TRY(cudaMemcpyAsync(d_idx, index_nodes, sizeof(int32_t) * n_index, cudaMemcpyHostToDevice, cs));
    }
    C_TRY(fs::launch_pack_init(e->d_X, (int)n, Rp, n_real, d_idx, n_index, g->d_inv, params[0].index_state,
                               e->d_mask[0], cs));
    if (e->push) {
        const size_t nt = (size_t)g->n_thr * Rp, nm = (size_t)std::max(g->n_m, 1) * Rp;
        C_TRY(fsapi::ensure_out_csr(g, cs));
        C_TRY(dev_alloc(&e->d_pc8, nt, &e->bytes));
        C_TRY(dev_alloc(&e->d_phc, nm, &e->bytes));
        C_TRY(cudaMemsetAsync(e->d_pc8, 0, std::max<size_t>(nt, 1), cs));
        C_TRY(cudaMemsetAsync(e->d_phc, 0, sizeof(uint32_t) * nm, cs));
        for (int q = 0; q < 2; ++q) {
            C_TRY(dev_alloc(&e->d_ppd[q], nt, &e->bytes));
            C_TRY(dev_alloc(&e->d_phpd[q], nm, &e->bytes));
            C_TRY(cudaMemsetAsync(e->d_ppd[q], 0, sizeof(uint16_t) * std::max<size_t>(nt, 1), cs));
            C_TRY(cudaMemsetAsync(e->d_phpd[q], 0, sizeof(unsigned long long) * nm, cs));
        }
        Member m0{e, 0, 0, nullptr};
        C_TRY(fs::launch_pack_push_init(segment_of(m0), cs));
    }
    if (e->shed && n_index > 0 && params[0].index_state == FS_I) {
        Member m0{e, 0, 0, nullptr};
        C_TRY(fs::launch_pack_rho_init(segment_of(m0), e->age_dtype, 0u, cs));
    }
    std::vector<uint32_t> cnt((size_t)Rp * 4, 0u);
    for (int r = 0; r < Rp; ++r) {
        if (r < n_real) {
            cnt[r * 4 + FS_S] = (uint32_t)(n - n_index);
            cnt[r * 4 + params[0].index_state] += (uint32_t)n_index;
        } else {
            cnt[r * 4 + FS_R] = (uint32_t)n;
        }
    }
    C_TRY(cudaMemcpyAsync(e->d_counts, cnt.data(), sizeof(uint32_t) * Rp * 4, cudaMemcpyHostToDevice, cs));
    C_TRY(cudaStreamSynchronize(cs));
#undef C_TRY
    fs::dfree(d_idx);
    g->refs += 1;
    *out = e;
    return FS_OK;
}

fs_status fs_ens_get_state(fs_ens* e, int32_t r, uint8_t* state, void* age, int64_t* step)
{
    if (!e)
        return fail(FS_EINVAL, "fs_ens_get_state: NULL ensemble");
    if (e->failed)
        return fail(FS_ESTATE, "fs_ens_get_state: ensemble is in a failed state");
    if (r < 0 || r >= e->R)
        return fail(FS_EINVAL, "fs_ens_get_state: replicate %d out of range", r);
    if (e->batch)
        E_CUDA(e, cudaStreamSynchronize(e->batch->stream));
    E_CUDA(e, cudaStreamSynchronize(e->stream));
    if (step)
        *step = e->steps_done;
    const fs_graph* g = e->g;
    const int64_t n = g->n;
    std::vector<int32_t> perm;
    if (!g->identity && (state || age)) {
        perm.resize((size_t)n);
        E_CUDA(e, cudaMemcpy(perm.data(), g->d_perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    }
    auto fetch = [&](const void* dbase, void* hout, int eb) -> cudaError_t {
        std::vector<uint8_t> tmp((size_t)n * eb);
        cudaError_t err = cudaMemcpy2D(tmp.data(), eb, (const uint8_t*)dbase + (size_t)r * eb, (size_t)e->R_pad * eb,
                                       eb, (size_t)n, cudaMemcpyDeviceToHost);
        if (err != cudaSuccess)
            return err;
        uint8_t* o = static_cast<uint8_t*>(hout);
        if (perm.empty())
            memcpy(o, tmp.data(), tmp.size());
        else
            for (int64_t i = 0; i < n; ++i)
                memcpy(o + (size_t)perm[i] * eb, tmp.data() + (size_t)i * eb, eb);
        return cudaSuccess;
    };
    if (state)
        E_CUDA(e, fetch(e->d_X, state, 1));
    if (age)
        E_CUDA(e, fetch(e->d_A, age, e->age_bytes));
    return FS_OK;
}

fs_status fs_ens_pressure_get(const fs_ens* e, int32_t* pressure)
{
    if (!e || !pressure)
        return fail(FS_EINVAL, "fs_ens_pressure_get: NULL argument");
    *pressure = e->push ? FS_PRESSURE_PUSH : FS_PRESSURE_GATHER;
    return FS_OK;
}

fs_status fs_ens_time(fs_ens* e, double* elapsed, float* next_dt)
{
    if (!e)
        return fail(FS_EINVAL, "fs_ens_time: NULL ensemble");
    if (e->failed)
        return fail(FS_ESTATE, "fs_ens_time: ensemble is in a failed state");
    if (e->batch)
        E_CUDA(e, cudaStreamSynchronize(e->batch->stream));
    E_CUDA(e, cudaStreamSynchronize(e->stream));
    const int Rp = e->R_pad;
    std::vector<double> t((size_t)Rp, 0.0);
    std::vector<uint32_t> lam((size_t)3 * Rp, 0u);
    if (e->d_time) {
        E_CUDA(e, cudaMemcpy(t.data(), e->d_time, sizeof(double) * Rp, cudaMemcpyDeviceToHost));
        E_CUDA(e, cudaMemcpy(lam.data(), e->d_lam, sizeof(uint32_t) * 3 * Rp, cudaMemcpyDeviceToHost));
    }
    for (int r = 0; r < e->R; ++r) {
        const fs::PackScen& S = e->h_scen[(size_t)r];
        if (!e->d_time) {
            // fixed step: every step has the same size
            if (elapsed)
                elapsed[r] = (double)e->steps_done * (double)S.M.dt;
            if (next_dt)
                next_dt[r] = S.M.dt;
            continue;
        }
        if (elapsed)
            elapsed[r] = t[(size_t)r];
        if (next_dt) {
            // the same FP32 operations as the step: min(dt, eps / (lambda* + delta))
            float lp;
            const uint32_t bits = lam[(size_t)((e->steps_done + 2) % 3) * Rp + r];
            memcpy(&lp, &bits, sizeof(lp));
            next_dt[r] = std::min(S.M.dt, S.eps / (lp + S.delta));
        }
    }
    return FS_OK;
}

fs_status fs_ens_destroy(fs_ens* e)
{
    if (!e)
        return fail(FS_EINVAL, "fs_ens_destroy: NULL ensemble");
    if (e->batch)
        return fail(FS_EBUSY, "fs_ens_destroy: the ensemble is a live member of a batch");
    e->g->refs -= 1;
    free_ens(e);
    return FS_OK;
}

fs_status fs_batch_create(int32_t age_dtype, int32_t max_members, void* stream, fs_batch** out)
{
    g_err.clear();
    if (!out)
        return fail(FS_EINVAL, "fs_batch_create: NULL out");
    *out = nullptr;
    if (age_dtype < FS_AGE_F32 || age_dtype > FS_AGE_BF16)
        return fail(FS_EINVAL, "fs_batch_create: bad age_dtype");
    if (max_members < 1 || max_members > (1 << 20))
        return fail(FS_EINVAL, "fs_batch_create: max_members must be in [1, 2^20]");
    fs_batch* b = new fs_batch();
    b->age_dtype = age_dtype;
    b->cap = max_members;
    auto bail = [&](cudaError_t e) {
        free_batch(b);
        return fail(e == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA, "fs_batch_create: %s",
                    cudaGetErrorString(e));
    };
    cudaError_t e = cudaSuccess;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = dev_alloc(&b->d_seg, (size_t)max_members, nullptr);
    if (e == cudaSuccess) e = dev_alloc(&b->d_thr, (size_t)max_members + 1, nullptr);
    if (e == cudaSuccess) e = dev_alloc(&b->d_hub, (size_t)max_members + 1, nullptr);
    if (e == cudaSuccess) e = dev_alloc(&b->d_cls, fs::kPackClasses + 1, nullptr);
    if (e == cudaSuccess) e = dev_alloc(&b->d_ctl, 1, nullptr);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_seg, sizeof(fs::PackSeg) * max_members);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_thr, sizeof(int64_t) * (max_members + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_hub, sizeof(int64_t) * (max_members + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_cls, sizeof(int32_t) * (fs::kPackClasses + 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctl, 0, sizeof(fs::DevCtl), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_cls, 0, sizeof(int32_t) * (fs::kPackClasses + 1), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_thr, 0, sizeof(int64_t), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_hub, 0, sizeof(int64_t), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bail(e);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int c = 0; c < 3; ++c)
        b->grid[c] = fs::pack_grid(sms, c);
    *out = b;
    return FS_OK;
}

fs_status fs_batch_add(fs_batch* b, fs_ens* e, int64_t steps, uint32_t* counts_out)
{
    if (!b || !e)
        return fail(FS_EINVAL, "fs_batch_add: NULL argument");
    if (b->failed || e->failed)
        return fail(FS_ESTATE, "fs_batch_add: batch or ensemble in a failed state");
    if (e->batch)
        return fail(FS_EBUSY, "fs_batch_add: the ensemble is already a member of a batch");
    if (e->age_dtype != b->age_dtype)
        return fail(FS_EINVAL, "fs_batch_add: age_dtype differs from the batch's");
    if (steps < 0 || e->steps_done + steps >= ((int64_t)1 << 32))
        return fail(FS_EINVAL, "fs_batch_add: bad steps");
    if ((int32_t)b->members.size() >= b->cap)
        return fail(FS_ENOMEM, "fs_batch_add: the batch is full (%d members)", b->cap);
    if (counts_out) {
        const size_t bytes = sizeof(uint32_t) * (size_t)(steps + 1) * e->R_pad * 4;
        E_CUDA(e, fs::dmalloc(&e->d_out, bytes));
        E_CUDA(e, cudaStreamSynchronize(e->stream));
        E_CUDA(e, cudaMemcpyAsync(e->d_out, e->d_counts, sizeof(uint32_t) * e->R_pad * 4, cudaMemcpyDeviceToDevice,
                                  b->stream));
    }
    b->members.push_back(Member{e, b->G, steps, counts_out});
    e->batch = b;
    b->dirty = true;
    return FS_OK;
}

static int width_class(int R_pad)
{
    return R_pad == 8 ? 0 : R_pad == 16 ? 1 : 2;
}

static fs_status upload_table(fs_batch* b)
{
    E_CUDA(b, cudaStreamSynchronize(b->stream));     // the staging buffers are free again
    b->h_thr[0] = 0;
    b->h_hub[0] = 0;
    b->classes = 0;
    int q = 0;
    for (int c = 0; c < fs::kPackClasses; ++c) {      // rows ordered by replicate width, form, step
        b->h_cls[c] = q;
        for (const Member& m : b->members) {
            const int form = m.e->push ? 1 : m.e->shed ? 2 : 0;
            if ((width_class(m.e->R_pad) * 3 + form) * 2 + (m.e->d_lam ? 1 : 0) != c)
                continue;
            b->h_seg[q] = segment_of(m);
            const fs_graph* g = m.e->g;
            b->h_thr[q + 1] = b->h_thr[q] + (int64_t)g->n_slices;
            b->h_hub[q + 1] = b->h_hub[q] + g->n_m;
            b->classes |= 1 << c;
            ++q;
        }
    }
    b->h_cls[fs::kPackClasses] = q;
    const int ns = q;
    if (ns > 0)
        E_CUDA(b, cudaMemcpyAsync(b->d_seg, b->h_seg, sizeof(fs::PackSeg) * ns, cudaMemcpyHostToDevice, b->stream));
    E_CUDA(b, cudaMemcpyAsync(b->d_thr, b->h_thr, sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, b->stream));
    E_CUDA(b, cudaMemcpyAsync(b->d_hub, b->h_hub, sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, b->stream));
    E_CUDA(b, cudaMemcpyAsync(b->d_cls, b->h_cls, sizeof(int32_t) * (fs::kPackClasses + 1), cudaMemcpyHostToDevice,
                              b->stream));
    b->dirty = false;
    return FS_OK;
}

static fs::PackArgs pack_args(const fs_batch* b, int j)
{
    fs::PackArgs a{};
    a.seg = b->d_seg;
    a.thr_pre = b->d_thr;
    a.hub_pre = b->d_hub;
    a.cls = b->d_cls;
    a.ctl = b->d_ctl;
    a.j = j;
    return a;
}

// one step of every (width, form, step) class present in the table
static cudaError_t launch_classes(const fs_batch* b, int j, int classes)
{
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < fs::kPackClasses && e == cudaSuccess; ++c)
        if (classes & (1 << c))
            e = fs::launch_pack_step(pack_args(b, j), c / 6, (c / 2) % 3, (c & 1) != 0, b->age_dtype, b->grid[c / 6],
                                     b->stream);
    return e;
}

fs_status fs_batch_run(fs_batch* b, int64_t launches, int32_t graph_steps)
{
    if (!b)
        return fail(FS_EINVAL, "fs_batch_run: NULL batch");
    if (b->failed)
        return fail(FS_ESTATE, "fs_batch_run: batch in a failed state");
    const int K = graph_steps == 0 ? 50 : graph_steps;
    if (launches < 0 || K < 1 || K > fs::kMaxGraphSteps)
        return fail(FS_EINVAL, "fs_batch_run: bad launches or graph_steps");
    if (b->dirty) {
        fs_status st = upload_table(b);
        if (st != FS_OK)
            return st;
    }
    const int64_t full = launches / K;
    const int rem = (int)(launches % K);
    const int classes = b->classes;
    const int n_cls = __builtin_popcount((unsigned)classes);
    if (full > 0 && !(b->gexec && b->gK == K && b->g_classes == classes)) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        E_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int j = 0; j < K && e == cudaSuccess; ++j)
            e = launch_classes(b, j, classes);
        if (e == cudaSuccess)
            e = fs::launch_pack_advance(b->d_ctl, K, b->stream);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        E_CUDA(b, e);
        E_CUDA(b, e2);
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        E_CUDA(b, e);
        b->gK = K;
        b->g_classes = classes;
    }
    for (int64_t r = 0; r < full; ++r)
        E_CUDA(b, cudaGraphLaunch(b->gexec, b->stream));
    fs::g_launch_count += (unsigned long long)full * ((unsigned long long)K * n_cls + 1);
    if (rem > 0) {
        for (int j = 0; j < rem; ++j)
            E_CUDA(b, launch_classes(b, j, classes));
        E_CUDA(b, fs::launch_pack_advance(b->d_ctl, rem, b->stream));
    }
    b->G += launches;
    E_CUDA(b, cudaStreamSynchronize(b->stream));
    fs::DevCtl c;
    E_CUDA(b, cudaMemcpy(&c, b->d_ctl, sizeof(c), cudaMemcpyDeviceToHost));
    if (c.error) {
        b->failed = true;
        return fail(c.error == fs::kErrTmaTimeout ? FS_ETIMEOUT : FS_ECUDA, "fs_batch_run: device error word %d",
                    c.error);
    }
    // retire members whose last step has been integrated (at global step
    // g_join + steps, which must have been launched)
    std::vector<Member> keep;
    for (const Member& m : b->members) {
        if (m.g_join + m.steps < b->G) {
            fs_ens* e = m.e;
            if (m.host_out && e->d_out) {
                const size_t rows = (size_t)m.steps + 1;
                std::vector<uint32_t> tmp(rows * e->R_pad * 4);
                E_CUDA(b, cudaMemcpy(tmp.data(), e->d_out, sizeof(uint32_t) * tmp.size(), cudaMemcpyDeviceToHost));
                for (size_t row = 0; row < rows; ++row)
                    memcpy(m.host_out + row * e->R * 4, tmp.data() + row * e->R_pad * 4,
                           sizeof(uint32_t) * e->R * 4);
            }
            fs::dfree(e->d_out);
            e->d_out = nullptr;
            e->steps_done += m.steps;
            e->batch = nullptr;
            b->dirty = true;
        } else {
            keep.push_back(m);
        }
    }
    b->members.swap(keep);
    return FS_OK;
}

fs_status fs_batch_status(const fs_batch* b, int32_t* live, int64_t* launches_to_finish)
{
    if (!b)
        return fail(FS_EINVAL, "fs_batch_status: NULL batch");
    if (live)
        *live = (int32_t)b->members.size();
    if (launches_to_finish) {
        int64_t need = 0;
        for (const Member& m : b->members)
            need = std::max(need, m.g_join + m.steps + 1 - b->G);
        *launches_to_finish = need;
    }
    return FS_OK;
}

fs_status fs_batch_destroy(fs_batch* b)
{
    if (!b)
        return fail(FS_EINVAL, "fs_batch_destroy: NULL batch");
    cudaStreamSynchronize(b->stream);
    for (const Member& m : b->members) {
        fs::dfree(m.e->d_out);
        m.e->d_out = nullptr;
        m.e->batch = nullptr;
    }
    free_batch(b);
    return FS_OK;
}

fs_status fs_ens_run(fs_ens* e, int64_t steps, int32_t graph_steps, uint32_t* counts_out)
{
    if (!e)
        return fail(FS_EINVAL, "fs_ens_run: NULL ensemble");
    if (e->batch)
        return fail(FS_EBUSY, "fs_ens_run: the ensemble is a live member of a batch");
    fs_batch* b = nullptr;
    fs_status st = fs_batch_create(e->age_dtype, 1, e->stream, &b);
    if (st != FS_OK)
        return st;
    st = fs_batch_add(b, e, steps, counts_out);
    if (st == FS_OK)
        st = fs_batch_run(b, steps + 1, graph_steps);
    fs_batch_destroy(b);
    return st;
}

}  // extern "C"
