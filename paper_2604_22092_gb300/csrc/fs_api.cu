// fs_api.cu -- the C ABI of libflashstep (declared in include/fs.h): graph
// ingest orchestration, simulation state, and the step loop as CUDA Graph
// replays (FlashSpread, arXiv 2604.22092, Algorithm 2: capture of b steps with
// a persistent device step counter; Algorithm 3: the fused step).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fs.h"
#include "fs_launch.h"
#include "fs_objects.h"

namespace fsapi {

thread_local std::string g_err;

// failure-detection test settings (fs_test_inject), copied into every sim
// created while they are set
std::atomic<uint32_t> g_test_wait_limit{0};
std::atomic<int64_t> g_test_bounds_shrink{0};

fs_status fail(fs_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

}  // namespace fsapi

using fsapi::fail;
using fsapi::g_err;

#define FS_CUDA(obj, expr)                                                                     \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            if (obj)                                                                           \
                (obj)->failed = true;                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA, "%s: %s (%s:%d)", #expr, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                           \
        }                                                                                      \
    } while (0)

namespace fsapi {


void free_graph(fs_graph* g)
{
    if (!g)
        return;
    fs::dfree(g->d_perm);
    fs::dfree(g->d_inv);
    fs::dfree(g->d_deg);
    fs::dfree(g->d_sell_off);
    fs::dfree(g->d_sell_col);
    fs::dfree(g->d_m_ptr);
    fs::dfree(g->d_m_col);
    fs::dfree(g->d_m_warp_row);
    fs::dfree(g->d_m_chunk_last);
    fs::dfree(g->d_out_ptr);          // the columns share its allocation
    delete g;
}

void free_sim(fs_sim* s)
{
    if (!s)
        return;
    if (s->gexec)
        cudaGraphExecDestroy(s->gexec);
    fs::dfree(s->d_arena);          // every per-sim buffer but the counts output
    fs::dfree(s->d_counts);
    if (s->own_stream && s->stream)
        cudaStreamDestroy(s->stream);
    delete s;
}

bool finite(double v) { return std::isfinite(v); }

fs_status check_law(const fs_law& L, const char* what, bool allow_none)
{
    switch (L.kind) {
    case FS_LAW_NONE:
        if (!allow_none)
            return fail(FS_EINVAL, "%s law: kind NONE is not allowed here", what);
        return FS_OK;
    case FS_LAW_EXP:
        if (!finite(L.a) || L.a < 0)
            return fail(FS_EINVAL, "%s law: exponential rate must be finite and >= 0", what);
        return FS_OK;
    case FS_LAW_LOGNORMAL:
        if (!finite(L.a) || !finite(L.b) || !(L.b > 0))
            return fail(FS_EINVAL, "%s law: log-normal needs finite mu and sigma > 0", what);
        return FS_OK;
    case FS_LAW_WEIBULL:
        if (!finite(L.a) || !finite(L.b) || !(L.a >= 1.0) || !(L.b > 0))
            return fail(FS_EINVAL, "%s law: Weibull needs shape >= 1 and scale > 0", what);
        return FS_OK;
    case FS_LAW_ERLANG:
        if (L.k < 1 || L.k > 64 || !finite(L.a) || !(L.a > 0))
            return fail(FS_EINVAL, "%s law: Erlang needs 1 <= k <= 64 and rate > 0", what);
        return FS_OK;
    default:
        return fail(FS_EINVAL, "%s law: unknown kind %d", what, L.kind);
    }
}

fs::LawF to_lawf(const fs_law& L)
{
    fs::LawF f{};
    f.kind = L.kind;
    f.k = L.k;
    switch (L.kind) {
    case FS_LAW_EXP:
        f.p0 = (float)L.a;
        break;
    case FS_LAW_LOGNORMAL: {
        const double inv = 1.0 / (L.b * std::sqrt(2.0));
        f.p0 = (float)L.a;
        f.p3 = (float)(L.a - (double)f.p0);
        f.p1 = (float)inv;
        f.p4 = (float)(inv - (double)f.p1);
        f.p2 = (float)(std::sqrt(2.0 / M_PI) / L.b);
        break;
    }
    case FS_LAW_WEIBULL:
        f.p0 = (float)(L.a / L.b);
        f.p1 = (float)(1.0 / L.b);
        f.p2 = (float)(L.a - 1.0);
        break;
    case FS_LAW_ERLANG:
        f.p0 = (float)L.a;
        break;
    default:
        break;
    }
    return f;
}

fs_status check_params(const fs_sim_params* p)
{
    if (!p)
        return fail(FS_EINVAL, "params is NULL");
    if (p->model != FS_SIR && p->model != FS_SEIR && p->model != FS_SIS)
        return fail(FS_EINVAL, "model must be FS_SIR, FS_SEIR or FS_SIS");
    if (!finite(p->theta) || p->theta < 0 || !finite(p->p_max) || p->p_max < 0 || p->p_max > 1)
        return fail(FS_EINVAL, "theta must be finite and >= 0, p_max in [0, 1]");
    if (p->markov_mode < 0 || p->markov_mode > 2 || p->reserved2_ != 0)
        return fail(FS_EINVAL, "markov_mode must be 0, 1 or 2 and reserved2_ 0");
    if (p->theta > 0) {
        if (p->infectious.kind != FS_LAW_EXP || (p->model == FS_SEIR && p->latent.kind != FS_LAW_EXP))
            return fail(FS_EINVAL, "the Markovian engine (theta > 0) needs FS_LAW_EXP holding times");
        if (p->eps > 0 || p->shed_mode != FS_SHED_NONE || (p->flags & FS_ACTIVE_LIST))
            return fail(FS_EUNSUPPORTED, "the Markovian engine runs without eps, shedding and FS_ACTIVE_LIST");
    } else if (p->model == FS_SIS) {
        return fail(FS_EUNSUPPORTED, "FS_SIS runs in the Markovian engine (theta > 0)");
    }
    if (p->age_dtype < FS_AGE_F32 || p->age_dtype > FS_AGE_BF16)
        return fail(FS_EINVAL, "age_dtype must be FS_AGE_F32, FS_AGE_F16 or FS_AGE_BF16");
    if (!finite(p->beta) || p->beta < 0)
        return fail(FS_EINVAL, "beta must be finite and >= 0");
    if (!finite(p->dt) || !(p->dt > 0))
        return fail(FS_EINVAL, "dt must be finite and > 0");
    if ((p->flags & ~(FS_PRESSURE_MASK | FS_ACTIVE_LIST)) != 0 || (p->flags & FS_PRESSURE_MASK) > FS_PRESSURE_PUSH)
        return fail(FS_EINVAL, "flags must be FS_PRESSURE_AUTO, FS_PRESSURE_GATHER or FS_PRESSURE_PUSH, "
                               "optionally with FS_ACTIVE_LIST");
    if (p->shed_mode < FS_SHED_NONE || p->shed_mode > FS_SHED_DENSITY)
        return fail(FS_EINVAL, "shed_mode must be FS_SHED_NONE, FS_SHED_HAZARD or FS_SHED_DENSITY");
    if (p->shed_mode != FS_SHED_NONE) {
        fs_status st = check_law(p->shedding, "shedding", false);
        if (st != FS_OK)
            return st;
    }
    if (!finite(p->eps) || p->eps < 0 || !finite(p->delta) || p->delta < 0)
        return fail(FS_EINVAL, "eps and delta must be finite and >= 0");
    fs_status st = check_law(p->infectious, "infectious", false);
    if (st != FS_OK)
        return st;
    if (p->model == FS_SEIR) {
        st = check_law(p->latent, "latent", false);
        if (st != FS_OK)
            return st;
        if (p->index_state != FS_E && p->index_state != FS_I)
            return fail(FS_EINVAL, "SEIR index_state must be FS_E or FS_I");
    } else if (p->index_state != FS_I) {
        return fail(FS_EINVAL, "SIR index_state must be FS_I");
    }
    return FS_OK;
}

fs::ModelF to_model(const fs_sim_params& p)
{
    fs::ModelF M{};
    M.model = p.model;
    M.beta = (float)p.beta;
    M.dt = (float)p.dt;
    M.inv_dt = (float)(1.0 / p.dt);
    M.key0 = (uint32_t)(p.seed & 0xffffffffu);
    M.key1 = (uint32_t)(p.seed >> 32);
    M.rep = p.replicate;
    M.lat = to_lawf(p.latent);
    M.inf = to_lawf(p.infectious);
    return M;
}

fs::StepArgs step_args(const fs_sim* s, int j)
{
    const fs_graph* g = s->g;
    fs::StepArgs a{};
    a.X = s->d_X;
    a.A = s->d_A;
    a.bm[0] = s->d_bm[0];
    a.bm[1] = s->d_bm[1];
    a.sell_off = g->d_sell_off;
    a.sell_col = g->d_sell_col;
    a.n_thr = g->n_thr;
    a.n_slices = g->n_slices;
    a.sentinel = (int32_t)g->n;
    a.m_base = g->n_thr;
    a.n_m = g->n_m;
    a.n_chunks = g->n_chunks;
    a.m_ptr = g->d_m_ptr;
    a.m_col = g->d_m_col;
    a.m_warp_row = g->d_m_warp_row;
    a.m_chunk_last = g->d_m_chunk_last;
    a.e_m = g->e_m;
    a.m_cnt = s->d_m_cnt;
    a.m_tkt = s->d_m_tkt;
    a.perm = g->d_perm;
    a.deg = g->d_deg;
    a.ptab = s->d_ptab;
    a.ps = s->d_ps;
    a.spw = g->spw;
    a.n_sell_ctas = (g->n_slices + fs::kSellSlicesPerCta * g->spw - 1) / (fs::kSellSlicesPerCta * g->spw);
    a.bm_bytes = g->bm_bytes;
    a.smem_min_s = g->smem_min_s;
    a.M = s->M;
    a.ctl = s->d_ctl;
    a.deltas = s->d_deltas;
    a.j = j;
    a.n = (int32_t)g->n;
    a.cnt8 = s->d_cnt8;
    a.pd16[0] = s->d_pd16[0];
    a.pd16[1] = s->d_pd16[1];
    a.hcnt = s->d_hcnt;
    a.pd64[0] = s->d_pd64[0];
    a.pd64[1] = s->d_pd64[1];
    a.out_ptr = g->d_out_ptr;
    a.out_col = g->d_out_col;
    a.eps = (float)s->p.eps;
    a.delta = (float)(s->p.delta > 0 ? s->p.delta : 1e-12);
    a.rho[0] = s->d_rho[0];
    a.rho[1] = s->d_rho[1];
    a.m_part = s->d_mpart;
    a.shed = to_lawf(s->p.shedding);
    a.shed_mode = s->p.shed_mode;
    a.rtab = s->d_rtab;
    a.act = s->d_act;
    a.mk_cnt = s->d_mk_cnt;
    a.mk_ev = s->d_mk_ev;
    a.mk_beta = s->p.beta;
    a.mk_sigma = s->p.model == FS_SEIR ? s->p.latent.a : 0.0;
    a.mk_gamma = s->p.infectious.a;
    a.mk_theta = s->p.theta;
    a.mk_p_max = s->p.p_max > 0 ? s->p.p_max : 0.1;
    a.mk_tau_max = s->p.dt;
    a.mk_avg_deg = g->n ? (double)g->nnz / (double)g->n : 0.0;
    a.e_total = g->nnz;
    a.mk_mode = s->p.markov_mode;
    a.dtrec = s->d_dtrec;
    a.wait_limit = s->test_wait_limit;
    a.skip_bulk_copy = s->test_wait_limit ? 1 : 0;
    a.x_len = (g->n + 15) / 16 * 16 + 16;
    a.out_nnz = g->d_out_col ? g->nnz : 0;
    a.dbg_shrink = s->test_bounds_shrink;
    a.sell_len = g->sell_entries;
    a.bm_words = (g->n >> 5) + 1;
    return a;
}

// the push form needs u8 counts for the whole one-thread-per-node class
bool push_available(const fs_graph* g)
{
    return g->n_thr == 0 || g->t1 <= fs::kMaxThreadDeg;
}

// transposed CSR of the graph in internal ids (once per graph)
cudaError_t ensure_out_csr(fs_graph* g, cudaStream_t st)
{
    // graphs are shared by sims and by the server's thread
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (g->d_out_ptr)
        return cudaSuccess;
    const int64_t n = g->n;
    int64_t* optr = nullptr;
    int32_t* ocol = nullptr;
    unsigned long long* cur = nullptr;
    // row bounds and columns in one allocation (freed through d_out_ptr)
    const size_t ptr_bytes = ((sizeof(int64_t) * ((size_t)n + 1)) + 255) & ~(size_t)255;
    const int64_t bytes = (int64_t)(ptr_bytes + sizeof(int32_t) * std::max<int64_t>(g->nnz, 1));
    cudaError_t e = fs::dmalloc(reinterpret_cast<void**>(&optr), (size_t)bytes);
    if (e == cudaSuccess) {
        ocol = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(optr) + ptr_bytes);
        e = scratch_alloc(&cur, (size_t)n + 1, st);
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(cur, 0, sizeof(unsigned long long) * (n + 1), st);
    if (e == cudaSuccess)
        e = fs::launch_transpose(g->d_sell_off, g->d_sell_col, g->d_deg, g->n_thr, g->d_m_ptr, g->d_m_col, g->n_m,
                                 (int)n, cur, nullptr, false, st);
    if (e == cudaSuccess)
        e = fs::exclusive_scan_i64(reinterpret_cast<const int64_t*>(cur), optr, n, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cur, optr, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = fs::launch_transpose(g->d_sell_off, g->d_sell_col, g->d_deg, g->n_thr, g->d_m_ptr, g->d_m_col, g->n_m,
                                 (int)n, cur, ocol, true, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    scratch_free(cur, st);
    if (e != cudaSuccess) {
        fs::dfree(optr);
        return e;
    }
    g->d_out_ptr = optr;
    g->d_out_col = ocol;
    g->bytes += bytes;
    return cudaSuccess;
}

// counts and pending tallies of a push-form sim from its current state
cudaError_t push_reset(fs_sim* s)
{
    const fs_graph* g = s->g;
    const size_t thr_pad = ((size_t)g->n_thr + 15) / 16 * 16 + 16;
    cudaStream_t cs = s->stream;
    cudaError_t e = cudaMemsetAsync(s->d_cnt8, 0, thr_pad, cs);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q)
        e = cudaMemsetAsync(s->d_pd16[q], 0, thr_pad * sizeof(uint16_t), cs);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->d_hcnt, 0, sizeof(uint32_t) * std::max(g->n_m, 1), cs);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q)
        e = cudaMemsetAsync(s->d_pd64[q], 0, sizeof(unsigned long long) * std::max(g->n_m, 1), cs);
    if (e == cudaSuccess)
        e = fs::launch_push_init(step_args(s, 0), cs, g->num_sms);
    return e;
}

fs_status check_device_error(fs_sim* s)
{
    fs::DevCtl c;
    FS_CUDA(s, cudaMemcpy(&c, s->d_ctl, sizeof(c), cudaMemcpyDeviceToHost));
    if (c.error) {
        s->failed = true;
        if (c.error == fs::kErrTmaTimeout)
            return fail(FS_ETIMEOUT, "a bounded device wait ran out (error word %d)", c.error);
        if (c.error == fs::kErrBounds)
            return fail(FS_ECUDA, "bounds check failed: site %d, index %lld (error word %d)", c.dbg_site,
                        (long long)c.dbg_index, c.error);
        return fail(FS_ECUDA, "device error word %d", c.error);
    }
    return FS_OK;
}

}  // namespace fsapi

using namespace fsapi;

extern "C" {

const char* fs_version(void) { return "flashstep 0.1 sm_103a"; }

const char* fs_last_error(void) { return g_err.c_str(); }

fs_status fs_graph_create(int64_t n, const int64_t* row_ptr, const int32_t* col_ind, const float* weights,
                          const fs_graph_opts* opts, void* stream, fs_graph** out)
{
    g_err.clear();
    if (!out)
        return fail(FS_EINVAL, "out is NULL");
    *out = nullptr;
    fs_graph_opts o{};
    if (opts)
        o = *opts;
    if (weights)
        return fail(FS_EUNSUPPORTED, "edge weights are not supported (unit weights only)");
    if (n < 1 || n >= (int64_t)INT32_MAX)
        return fail(FS_EINVAL, "n must be in [1, 2^31 - 1)");
    if (!row_ptr)
        return fail(FS_EINVAL, "row_ptr is NULL");
    if (o.dispatch < FS_DISPATCH_AUTO || o.dispatch > FS_DISPATCH_TUNE)
        return fail(FS_EINVAL, "unknown dispatch %d", o.dispatch);
    if (o.dispatch == FS_DISPATCH_TUNE && o.thread_max_deg != 0)
        return fail(FS_EINVAL, "FS_DISPATCH_TUNE chooses thread_max_deg itself (pass 0)");
    if (o.thread_max_deg != 0 && (o.thread_max_deg < 31 || o.thread_max_deg > fs::kMaxThreadDeg))
        return fail(FS_EINVAL, "thread_max_deg must be 0 or in [31, %d]", fs::kMaxThreadDeg);
    if (o.device_input != 0 && o.device_input != 1)
        return fail(FS_EINVAL, "device_input must be 0 or 1");
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev_in = o.device_input == 1;
    int64_t nnz = 0;
    if (!dev_in) {
        // the rows' monotonicity and the column range are checked on the
        // device after the copy (as for device input), not by host loops
        if (row_ptr[0] != 0)
            return fail(FS_EINVAL, "row_ptr[0] must be 0");
        nnz = row_ptr[n];
        if (nnz < 0)
            return fail(FS_EINVAL, "row_ptr[n] < 0");
        if (nnz > 0 && !col_ind)
            return fail(FS_EINVAL, "col_ind is NULL");
    } else {
        cudaError_t e = cudaMemcpy(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return fail(FS_ECUDA, "reading row_ptr[n]: %s", cudaGetErrorString(e));
        if (nnz < 0)
            return fail(FS_EINVAL, "row_ptr[n] < 0");
        if (nnz > 0 && !col_ind)
            return fail(FS_EINVAL, "col_ind is NULL");
    }
    if (o.dispatch == FS_DISPATCH_TUNE) {
        // the degree profile first (d_max), then the tuner builds what it needs
        int64_t dmax = 0;
        if (!dev_in) {
            for (int64_t i = 0; i < n; ++i)
                dmax = std::max(dmax, row_ptr[i + 1] - row_ptr[i]);
        } else {
            fs::IngestFlags* d_fl = nullptr;
            fs::IngestFlags hf{};
            cudaError_t e = dev_alloc(&d_fl, 1, nullptr);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(d_fl, 0, sizeof(fs::IngestFlags), st);
            if (e == cudaSuccess)
                e = fs::launch_degrees(row_ptr, (int)n, fs::kMaxThreadDeg, nullptr, nullptr, d_fl, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&hf, d_fl, sizeof(hf), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(st);
            fs::dfree(d_fl);
            if (e != cudaSuccess)
                return fail(FS_ECUDA, "degree profile: %s", cudaGetErrorString(e));
            if (hf.error)
                return fail(FS_EINVAL, "row_ptr is not a valid CSR row pointer");
            dmax = hf.dmax;
        }
        fs_graph_opts a = o;
        a.dispatch = FS_DISPATCH_AUTO;
        return fsapi::tune_create(n, nnz, dmax, row_ptr, col_ind, a, stream, out);
    }

    fs_graph* g = new fs_graph();
    g->n = n;
    g->nnz = nnz;
    fs_status rc = FS_OK;
    const int ni = (int)n;
    int64_t* d_rp = nullptr;
    int32_t* d_col = nullptr;
    uint16_t* d_key = nullptr;
    fs::IngestFlags* d_flags = nullptr;
    int64_t* d_tmp = nullptr;
    fs::IngestFlags fl{};
    auto cleanup = [&]() {
        if (!dev_in) {
            fs::dfree(d_rp);
            fs::dfree(d_col);
        }
        scratch_free(d_key, st);
        scratch_free(d_flags, st);
        scratch_free(d_tmp, st);
    };
#define G_CUDA(expr)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            rc = fail(e_ == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA, "%s: %s", #expr,       \
                      cudaGetErrorString(e_));                                                        \
            goto done;                                                                                \
        }                                                                                             \
    } while (0)
    {
        if (dev_in) {
            d_rp = const_cast<int64_t*>(row_ptr);
            d_col = const_cast<int32_t*>(col_ind);
        } else {
            G_CUDA(dev_alloc(&d_rp, (size_t)n + 1, nullptr));
            G_CUDA(dev_alloc(&d_col, (size_t)nnz, nullptr));
            G_CUDA(cudaMemcpyAsync(d_rp, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
            if (nnz)
                G_CUDA(cudaMemcpyAsync(d_col, col_ind, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
        }
        G_CUDA(dev_alloc(&g->d_deg, (size_t)n, &g->bytes));
        G_CUDA(scratch_alloc(&d_key, (size_t)n, st));
        G_CUDA(scratch_alloc(&d_flags, 1, st));
        // pass 1: degrees, d_max, validity
        G_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(fs::IngestFlags), st));
        G_CUDA(fs::launch_degrees(d_rp, ni, fs::kMaxThreadDeg, g->d_deg, d_key, d_flags, st));
        G_CUDA(fs::launch_check_cols(d_col, nnz, ni, d_flags, st));
        G_CUDA(cudaMemcpyAsync(&fl, d_flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
        G_CUDA(cudaStreamSynchronize(st));
        if (fl.error) {
            rc = fail(FS_EINVAL, fl.error == 2 ? "col_ind out of range" : "row_ptr is not a valid CSR row pointer");
            goto done;
        }
        g->dmax = fl.dmax;
        // class threshold (Section 5.5 auto-dispatch, adapted: a degree split)
        bool all_thread = false;
        if (o.dispatch == FS_DISPATCH_THREAD) {
            all_thread = true;
        } else if (o.dispatch == FS_DISPATCH_MERGE) {
            g->t1 = fs::kMinMergeDegree - 1;
        } else if (o.thread_max_deg > 0) {
            g->t1 = o.thread_max_deg;
        } else {
            g->t1 = (g->dmax <= 64) ? g->dmax : 63;
        }
        if (all_thread) {
            g->t1 = g->dmax;
            g->n_thr = ni;
            g->identity = true;
        } else if (g->t1 >= g->dmax) {
            // every node is in the thread class and the first pass's keys (the
            // degrees, all <= 255) are this split's keys: no second pass
            g->n_thr = ni;
            g->identity = fl.unsorted == 0;
        } else {
            G_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(fs::IngestFlags), st));
            G_CUDA(fs::launch_degrees(d_rp, ni, g->t1, g->d_deg, d_key, d_flags, st));
            G_CUDA(cudaMemcpyAsync(&fl, d_flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
            G_CUDA(cudaStreamSynchronize(st));
            g->n_thr = fl.n_thr;
            g->identity = fl.unsorted == 0;
        }
        g->n_m = ni - g->n_thr;
        if (!g->identity) {
            int32_t* deg_int = nullptr;
            G_CUDA(dev_alloc(&g->d_perm, (size_t)n, &g->bytes));
            G_CUDA(dev_alloc(&g->d_inv, (size_t)n, &g->bytes));
            G_CUDA(dev_alloc(&deg_int, (size_t)n, nullptr));
            G_CUDA(fs::stable_sort_by_key(d_key, g->d_deg, ni, g->t1 + 2, g->d_perm, g->d_inv, deg_int, st));
            G_CUDA(cudaStreamSynchronize(st));
            fs::dfree(g->d_deg);
            g->d_deg = deg_int;
        }
        // SELL-32 blocks of the thread class; slices per warp so that the
        // step grid is about one wave of resident CTAs
        g->n_slices = (g->n_thr + 31) / 32;
        {
            int dev = 0, sms = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
                g->num_sms = sms;
            const int64_t wave_warps = (int64_t)g->num_sms * fs::kStepCtasPerSm * fs::kStepWarps;
            g->spw = (int32_t)std::max<int64_t>(1, (g->n_slices + wave_warps - 1) / wave_warps);
            // shared-memory bitmap path: the whole bitmap fits one CTA's shared
            // memory; it pays off once the S nodes' gathers outweigh one copy of
            // the bitmap per SM (about 4 gathers per node, measured)
            g->bm_bytes = (uint32_t)((((n >> 5) + 1) * 4 + 15) / 16 * 16);
            g->smem_path = g->n_slices > 0 && g->bm_bytes <= fs::kSmemBitmapMaxBytes;
            const double d_avg = n ? (double)nnz / (double)n : 0.0;
            g->smem_min_s = (uint32_t)std::min<double>((double)n, 4.0 * (double)n / std::max(d_avg, 1.0));
        }
        G_CUDA(dev_alloc(&g->d_sell_off, (size_t)g->n_slices + 1, &g->bytes));
        G_CUDA(scratch_alloc(&d_tmp, (size_t)std::max(g->n_slices, g->n_m) + 1, st));
        G_CUDA(fs::launch_sell_widths(g->d_deg, g->n_thr, g->n_slices, d_tmp, st));
        G_CUDA(fs::exclusive_scan_i64(d_tmp, g->d_sell_off, g->n_slices, st));
        G_CUDA(cudaMemcpyAsync(&g->sell_entries, g->d_sell_off + g->n_slices, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, st));
        G_CUDA(cudaStreamSynchronize(st));
        G_CUDA(dev_alloc(&g->d_sell_col, (size_t)g->sell_entries, &g->bytes));
        G_CUDA(fs::launch_sell_fill(d_rp, d_col, g->d_perm, g->d_inv, g->d_deg, g->n_thr, g->n_slices,
                                    g->d_sell_off, (int)n, g->d_sell_col, st));
        // CSR and chunk tables of the merge class
        if (g->n_m > 0) {
            G_CUDA(dev_alloc(&g->d_m_ptr, (size_t)g->n_m + 1, &g->bytes));
            G_CUDA(fs::launch_merge_degrees(g->d_deg, g->n_thr, g->n_m, d_tmp, st));
            G_CUDA(fs::exclusive_scan_i64(d_tmp, g->d_m_ptr, g->n_m, st));
            G_CUDA(cudaMemcpyAsync(&g->e_m, g->d_m_ptr + g->n_m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            G_CUDA(cudaStreamSynchronize(st));
            const int64_t chunks = (g->e_m + fs::kMergeEPB - 1) / fs::kMergeEPB;
            if (chunks >= INT32_MAX) {
                rc = fail(FS_EUNSUPPORTED, "too many merge chunks");
                goto done;
            }
            g->n_chunks = (int32_t)chunks;
            const int64_t padded = chunks * fs::kMergeEPB;
            G_CUDA(dev_alloc(&g->d_m_col, (size_t)padded, &g->bytes));
            G_CUDA(fs::launch_merge_fill(d_rp, d_col, g->d_perm, g->d_inv, g->n_thr, g->n_m, g->d_m_ptr, g->e_m,
                                         padded, (int)n, g->d_m_col, st));
            G_CUDA(dev_alloc(&g->d_m_warp_row, (size_t)chunks * fs::kStepWarps, &g->bytes));
            G_CUDA(dev_alloc(&g->d_m_chunk_last, (size_t)chunks, &g->bytes));
            G_CUDA(fs::launch_merge_tables(g->d_m_ptr, g->n_m, g->e_m, g->n_chunks, g->d_m_warp_row,
                                           g->d_m_chunk_last, st));
        }
        G_CUDA(cudaStreamSynchronize(st));
    }
done:
#undef G_CUDA
    cleanup();
    if (rc != FS_OK) {
        free_graph(g);
        return rc;
    }
    *out = g;
    return FS_OK;
}

fs_status fs_graph_info(const fs_graph* g, fs_graph_info_t* out)
{
    if (!g || !out)
        return fail(FS_EINVAL, "NULL argument");
    fs_graph_info_t i{};
    i.n = g->n;
    i.nnz = g->nnz;
    i.d_max = g->dmax;
    i.d_avg = g->n ? (double)g->nnz / (double)g->n : 0.0;
    i.rho = i.d_avg > 0 ? (double)g->dmax / i.d_avg : 0.0;
    i.n_thread = g->n_thr;
    i.n_merge = g->n_m;
    i.sell_entries = g->sell_entries;
    i.merge_chunks = g->n_chunks;
    i.thread_max_deg = g->t1;
    i.identity_layout = g->identity ? 1 : 0;
    i.device_bytes = g->bytes;
    *out = i;
    return FS_OK;
}

fs_status fs_graph_info_get(const fs_graph* g, fs_graph_info_t* out)
{
    return fs_graph_info(g, out);
}

fs_status fs_graph_destroy(fs_graph* g)
{
    if (!g)
        return fail(FS_EINVAL, "graph is NULL");
    if (g->refs > 0)
        return fail(FS_EBUSY, "%d simulation(s) still use this graph", g->refs);
    free_graph(g);
    return FS_OK;
}

fs_status fs_sim_init(fs_graph* g, const fs_sim_params* params, const int32_t* index_nodes, int64_t n_index,
                      void* stream, fs_sim** out)
{
    g_err.clear();
    if (!g || !out)
        return fail(FS_EINVAL, "NULL argument");
    *out = nullptr;
    if (g->failed)
        return fail(FS_ESTATE, "graph is in a failed state");
    fs_status st = check_params(params);
    if (st != FS_OK)
        return st;
    if (n_index < 0 || n_index > g->n || (n_index > 0 && !index_nodes))
        return fail(FS_EINVAL, "bad index list size");
    {
        std::vector<int32_t> v(index_nodes, index_nodes + n_index);
        std::sort(v.begin(), v.end());
        for (int64_t q = 0; q < n_index; ++q) {
            if (v[q] < 0 || v[q] >= g->n)
                return fail(FS_EINVAL, "index node %d out of range", v[q]);
            if (q && v[q] == v[q - 1])
                return fail(FS_EINVAL, "index node %d repeated", v[q]);
        }
    }
    const bool markov = params->theta > 0;    // keeps its own exact counts: the pressure form is ignored
    const int pform = markov ? FS_PRESSURE_AUTO : (params->flags & FS_PRESSURE_MASK);
    if (pform == FS_PRESSURE_PUSH && !push_available(g))
        return fail(FS_EUNSUPPORTED, "FS_PRESSURE_PUSH needs in-degrees <= %d in the thread class (thread_max_deg %d)",
                    fs::kMaxThreadDeg, g->t1);
    const bool shed = params->shed_mode != FS_SHED_NONE;
    if (shed && pform == FS_PRESSURE_PUSH)
        return fail(FS_EUNSUPPORTED, "a shedding profile needs the gather form of the pressure (the push form "
                                     "keeps integer infectious counts)");
    fs_sim* s = new fs_sim();
    s->g = g;
    s->p = *params;
    s->test_wait_limit = g_test_wait_limit.load();
    s->test_bounds_shrink = g_test_bounds_shrink.load();
    s->pressure = (markov || shed || pform == FS_PRESSURE_GATHER || !push_available(g)) ? FS_PRESSURE_GATHER
                                                                                        : FS_PRESSURE_PUSH;
    s->markov = markov;
    s->M = to_model(*params);
    s->age_bytes = params->age_dtype == FS_AGE_F32 ? 4 : 2;
    const int64_t n = g->n;
    int32_t* d_idx = nullptr;
    auto bail = [&](fs_status rc) {
        free_sim(s);
        return rc;
    };
#define S_CUDA(expr)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA, "%s: %s", #expr, \
                             cudaGetErrorString(e_)));                                                \
    } while (0)
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        S_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        s->own_stream = true;
    }
    cudaStream_t cs = s->stream;
    const size_t words = ((size_t)(n >> 5) + 1 + 3) / 4 * 4;
    // whole 16-node groups (+16) for the vector accesses of the push step
    const size_t n_pad = ((size_t)n + 15) / 16 * 16 + 16;
    const size_t thr_pad = ((size_t)g->n_thr + 15) / 16 * 16 + 16;
    const size_t nm1 = (size_t)std::max(g->n_m, 1);
    const bool push = s->pressure == FS_PRESSURE_PUSH;
    // every buffer of the sim is carved from one allocation (256-byte aligned
    // pieces), zeroed by one memset
    size_t arena = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = arena;
        arena = (arena + std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
        return o;
    };
    const size_t oX = carve(n_pad), oA = carve(n_pad * s->age_bytes);
    const size_t oB0 = carve(words * 4), oB1 = carve(words * 4);
    const size_t oMc = carve(sizeof(int32_t) * nm1), oMt = carve(sizeof(uint32_t) * nm1);
    const size_t oCtl = carve(sizeof(fs::DevCtl));
    const size_t oDel = carve(sizeof(unsigned long long) * fs::kMaxGraphSteps * fs::kDeltaRow);
    const size_t oPt = carve(sizeof(float4) * 2 * fs::kPTableN), oPs = carve(sizeof(float) * fs::kPSTableN);
    const size_t oIdx = carve(sizeof(int32_t) * (size_t)std::max<int64_t>(n_index, 1));
    const size_t oDt = carve(sizeof(float) * fs::kMaxGraphSteps);
    const size_t oMkc = markov ? carve(sizeof(uint32_t) * n_pad) : 0;
    const size_t oMke = markov ? carve(sizeof(uint32_t) * n_pad) : 0;
    // active-node compaction list: one entry per push item or SELL slice
    const bool compact = (params->flags & FS_ACTIVE_LIST) != 0;
    const size_t n_units = push ? ((size_t)g->n_thr + fs::kPushG - 1) / fs::kPushG + (size_t)g->n_m
                                : (size_t)g->n_slices;
    const size_t oAct = compact ? carve(sizeof(int32_t) * (n_units + 32)) : 0;
    size_t oR0 = 0, oR1 = 0, oMp = 0, oRt = 0;
    if (shed) {
        oR0 = carve(n_pad * s->age_bytes);
        oR1 = carve(n_pad * s->age_bytes);
        oMp = carve(sizeof(float2) * (size_t)std::max(g->n_chunks, 1));
        oRt = carve(sizeof(float4) * fs::kPTableN);
    }
    size_t oC8 = 0, oP0 = 0, oP1 = 0, oHc = 0, oH0 = 0, oH1 = 0;
    if (push) {
        oC8 = carve(thr_pad);
        oP0 = carve(sizeof(uint16_t) * thr_pad);
        oP1 = carve(sizeof(uint16_t) * thr_pad);
        oHc = carve(sizeof(uint32_t) * nm1);
        oH0 = carve(sizeof(unsigned long long) * nm1);
        oH1 = carve(sizeof(unsigned long long) * nm1);
    }
    S_CUDA(fs::dmalloc(&s->d_arena, arena));
    char* base = static_cast<char*>(s->d_arena);
    s->d_X = reinterpret_cast<uint8_t*>(base + oX);
    s->d_A = base + oA;
    s->d_bm[0] = reinterpret_cast<uint32_t*>(base + oB0);
    s->d_bm[1] = reinterpret_cast<uint32_t*>(base + oB1);
    s->d_m_cnt = reinterpret_cast<int32_t*>(base + oMc);
    s->d_m_tkt = reinterpret_cast<uint32_t*>(base + oMt);
    s->d_ctl = reinterpret_cast<fs::DevCtl*>(base + oCtl);
    s->d_deltas = reinterpret_cast<unsigned long long*>(base + oDel);
    s->d_ptab = reinterpret_cast<float4*>(base + oPt);
    s->d_ps = reinterpret_cast<float*>(base + oPs);
    d_idx = reinterpret_cast<int32_t*>(base + oIdx);
    if (params->eps > 0 || markov)
        s->d_dtrec = reinterpret_cast<float*>(base + oDt);
    if (markov) {
        s->d_mk_cnt = reinterpret_cast<uint32_t*>(base + oMkc);
        s->d_mk_ev = reinterpret_cast<uint32_t*>(base + oMke);
    }
    if (compact)
        s->d_act = reinterpret_cast<int32_t*>(base + oAct);
    if (shed) {
        s->d_rho[0] = base + oR0;
        s->d_rho[1] = base + oR1;
        s->d_mpart = reinterpret_cast<float2*>(base + oMp);
        s->d_rtab = reinterpret_cast<float4*>(base + oRt);
    }
    if (push) {
        s->d_cnt8 = reinterpret_cast<uint8_t*>(base + oC8);
        s->d_pd16[0] = reinterpret_cast<uint16_t*>(base + oP0);
        s->d_pd16[1] = reinterpret_cast<uint16_t*>(base + oP1);
        s->d_hcnt = reinterpret_cast<uint32_t*>(base + oHc);
        s->d_pd64[0] = reinterpret_cast<unsigned long long*>(base + oH0);
        s->d_pd64[1] = reinterpret_cast<unsigned long long*>(base + oH1);
    }
    // all S, ages 0, bitmaps / scratch / control / deltas / counts / tallies 0
    S_CUDA(cudaMemsetAsync(s->d_arena, 0, arena, cs));
    S_CUDA(cudaMemsetAsync(s->d_ptab, 0xff, sizeof(float4) * 2 * fs::kPTableN, cs));   // NaN ages: no entry
    if (shed)
        S_CUDA(cudaMemsetAsync(s->d_rtab, 0xff, sizeof(float4) * fs::kPTableN, cs));
    S_CUDA(fs::launch_build_ptables(s->M, params->age_dtype, s->d_ptab, s->d_ps, cs, s->d_rtab,
                                    to_lawf(params->shedding), params->shed_mode));
    if (n_index > 0) {
        S_CUDA(cudaMemcpyAsync(d_idx, index_nodes, sizeof(int32_t) * n_index, cudaMemcpyHostToDevice, cs));
        S_CUDA(fs::launch_set_index(s->d_X, d_idx, n_index, g->d_inv, params->index_state, cs));
    }
    S_CUDA(fs::launch_refresh(s->d_X, (int)n, g->d_deg, s->d_bm[0], s->d_bm[1], s->d_ctl, cs));
    if (shed)
        S_CUDA(fs::launch_rho_init(step_args(s, 0), params->age_dtype, 0u, cs));
    if (markov) {
        S_CUDA(ensure_out_csr(g, cs));
        S_CUDA(fs::launch_markov_recount(step_args(s, 0), cs, g->num_sms));
    }
    if (push) {
        S_CUDA(ensure_out_csr(g, cs));
        S_CUDA(fs::launch_push_init(step_args(s, 0), cs, g->num_sms));   // counts and tallies are zero
    }
    S_CUDA(cudaStreamSynchronize(cs));
#undef S_CUDA
    g->refs += 1;
    *out = s;
    return FS_OK;
}

// one fused step: the shared-memory-bitmap grids when the bitmap fits, else
// the single mixed grid
static cudaError_t launch_one_step(fs_sim* s, int j)
{
    const fs::StepArgs a = step_args(s, j);
    if (s->markov)
        return fs::launch_markov_step(a, s->p.age_dtype, s->stream, s->g->num_sms);
    if (s->pressure == FS_PRESSURE_PUSH && s->d_dtrec)
        return fs::launch_push_step_adaptive(a, s->p.age_dtype, s->stream, s->g->num_sms);
    if (s->pressure == FS_PRESSURE_PUSH)
        return fs::launch_push_step(a, s->p.age_dtype, s->stream, s->g->num_sms);
    if (s->g->smem_path)
        return fs::launch_step_smem(a, s->p.age_dtype, s->stream, s->g->num_sms);
    return fs::launch_step(a, s->p.age_dtype, s->stream, false);
}

// the active-node compaction refresh that opens every launch sequence
static cudaError_t launch_compact(fs_sim* s)
{
    if (!s->d_act)
        return cudaSuccess;
    const fs::StepArgs a = step_args(s, 0);
    return s->pressure == FS_PRESSURE_PUSH ? fs::launch_push_compact(a, s->stream, s->g->num_sms)
                                           : fs::launch_sell_compact(a, s->stream, s->g->num_sms);
}

static fs_status ensure_graph(fs_sim* s, int K)
{
    if (s->gexec && s->gK == K)
        return FS_OK;
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    FS_CUDA(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_compact(s);
    for (int j = 0; j < K && e == cudaSuccess; ++j)
        e = launch_one_step(s, j);
    if (e == cudaSuccess)
        e = fs::launch_run_epilogue(s->d_ctl, s->d_deltas, K, s->p.model, s->d_dtrec, s->M.dt, s->stream);
    cudaError_t e2 = cudaStreamEndCapture(s->stream, &graph);
    FS_CUDA(s, e);
    FS_CUDA(s, e2);
    e = cudaGraphInstantiate(&s->gexec, graph, 0);
    cudaGraphDestroy(graph);
    FS_CUDA(s, e);
    s->gK = K;
    return FS_OK;
}

static fs_status run_enqueue(fs_sim* s, int64_t steps, int32_t graph_steps, uint32_t* counts_dev,
                             cudaEvent_t* replay_ev)
{
    if (!s)
        return fail(FS_EINVAL, "sim is NULL");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    if (steps < 0)
        return fail(FS_EINVAL, "steps must be >= 0");
    const int K = graph_steps == 0 ? 50 : graph_steps;
    if (K < 1 || K > fs::kMaxGraphSteps)
        return fail(FS_EINVAL, "graph_steps must be in [1, %d]", fs::kMaxGraphSteps);
    FS_CUDA(s, fs::launch_run_begin(s->d_ctl, counts_dev, s->stream));
    const int64_t full = steps / K;
    const int rem = (int)(steps % K);
    if (full > 0) {
        fs_status st = ensure_graph(s, K);
        if (st != FS_OK)
            return st;
        for (int64_t r = 0; r < full; ++r) {
            if (replay_ev)
                FS_CUDA(s, cudaEventRecord(replay_ev[r], s->stream));
            FS_CUDA(s, cudaGraphLaunch(s->gexec, s->stream));
        }
        fs::g_launch_count += (unsigned long long)full * ((s->markov ? 3 : 1) * K + 1 + (s->d_act ? 1 : 0));
    }
    if (replay_ev)
        FS_CUDA(s, cudaEventRecord(replay_ev[full], s->stream));
    if (rem > 0) {
        FS_CUDA(s, launch_compact(s));
        for (int j = 0; j < rem; ++j)
            FS_CUDA(s, launch_one_step(s, j));
        FS_CUDA(s, fs::launch_run_epilogue(s->d_ctl, s->d_deltas, rem, s->p.model, s->d_dtrec, s->M.dt, s->stream));
    }
    if (replay_ev)
        FS_CUDA(s, cudaEventRecord(replay_ev[full + 1], s->stream));
    return FS_OK;
}

fs_status fs_sim_run_async(fs_sim* s, int64_t steps, int32_t graph_steps, uint32_t* counts_dev)
{
    return run_enqueue(s, steps, graph_steps, counts_dev, nullptr);
}

fs_status fs_sim_run_timed(fs_sim* s, int64_t steps, int32_t graph_steps, uint32_t* counts_dev,
                            float* replay_ms, int64_t* n_replays)
{
    if (!s || !replay_ms || !n_replays)
        return fail(FS_EINVAL, "NULL argument");
    const int K = graph_steps == 0 ? 50 : graph_steps;
    if (K < 1 || K > fs::kMaxGraphSteps || steps < 0)
        return fail(FS_EINVAL, "bad steps or graph_steps");
    const int64_t full = steps / K;
    std::vector<cudaEvent_t> ev((size_t)full + 2, nullptr);
    for (auto& e : ev)
        FS_CUDA(s, cudaEventCreate(&e));
    fs_status st = run_enqueue(s, steps, graph_steps, counts_dev, ev.data());
    if (st == FS_OK)
        st = fs_sim_sync(s);
    if (st == FS_OK) {
        for (int64_t r = 0; r < full; ++r)
            cudaEventElapsedTime(&replay_ms[r], ev[r], ev[r + 1]);
        cudaEventElapsedTime(&replay_ms[full], ev[full], ev[full + 1]);
        *n_replays = full + 1;
    }
    for (auto& e : ev)
        cudaEventDestroy(e);
    return st;
}

fs_status fs_test_inject(int32_t what, int64_t value)
{
    g_err.clear();
    if (what == FS_TEST_WAIT_TIMEOUT) {
        if (value < 0 || value > (int64_t)fs::kWaitLimit)
            return fail(FS_EINVAL, "fs_test_inject: wait limit must be in [0, %u]", fs::kWaitLimit);
        g_test_wait_limit.store((uint32_t)value);
        return FS_OK;
    }
    if (what == FS_TEST_BOUNDS_SHRINK) {
#ifndef FS_DEBUG_BOUNDS
        return fail(FS_EUNSUPPORTED, "fs_test_inject: bounds checks exist only in the FS_DEBUG_BOUNDS build");
#else
        if (value < 0)
            return fail(FS_EINVAL, "fs_test_inject: shrink must be >= 0");
        g_test_bounds_shrink.store(value);
        return FS_OK;
#endif
    }
    return fail(FS_EINVAL, "fs_test_inject: unknown setting %d", what);
}

fs_status fs_debug_bounds_build(int32_t* enabled)
{
    if (!enabled)
        return fail(FS_EINVAL, "NULL argument");
#ifdef FS_DEBUG_BOUNDS
    *enabled = 1;
#else
    *enabled = 0;
#endif
    return FS_OK;
}

fs_status fs_kernel_launches(uint64_t* count)
{
    if (!count)
        return fail(FS_EINVAL, "NULL argument");
    *count = fs::g_launch_count.load();
    return FS_OK;
}

fs_status fs_sim_sync(fs_sim* s)
{
    if (!s)
        return fail(FS_EINVAL, "sim is NULL");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    FS_CUDA(s, cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

fs_status fs_sim_run(fs_sim* s, int64_t steps, int32_t graph_steps, uint32_t* counts_out)
{
    if (!s)
        return fail(FS_EINVAL, "sim is NULL");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    if (steps < 0)
        return fail(FS_EINVAL, "steps must be >= 0");
    uint32_t* dc = nullptr;
    if (counts_out) {
        const int64_t need = (steps + 1) * 4;
        if (need > s->counts_cap) {
            fs::dfree(s->d_counts);
            s->d_counts = nullptr;
            s->counts_cap = 0;
            FS_CUDA(s, fs::dmalloc(&s->d_counts, sizeof(uint32_t) * need));
            s->counts_cap = need;
        }
        dc = s->d_counts;
    }
    fs_status st = fs_sim_run_async(s, steps, graph_steps, dc);
    if (st != FS_OK)
        return st;
    if (counts_out)
        FS_CUDA(s, cudaMemcpyAsync(counts_out, dc, sizeof(uint32_t) * (steps + 1) * 4, cudaMemcpyDeviceToHost,
                                   s->stream));
    return fs_sim_sync(s);
}

fs_status fs_sim_step(fs_sim* s, uint32_t* counts_out)
{
    uint32_t c[8];
    fs_status st = fs_sim_run(s, 1, 1, c);
    if (st == FS_OK && counts_out)
        memcpy(counts_out, c + 4, sizeof(uint32_t) * 4);
    return st;
}

fs_status fs_sim_get_state(fs_sim* s, uint8_t* state, void* age, int64_t* step)
{
    if (!s)
        return fail(FS_EINVAL, "sim is NULL");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    const fs_graph* g = s->g;
    const int n = (int)g->n;
    FS_CUDA(s, cudaStreamSynchronize(s->stream));
    if (step) {
        fs::DevCtl c;
        FS_CUDA(s, cudaMemcpy(&c, s->d_ctl, sizeof(c), cudaMemcpyDeviceToHost));
        *step = c.step;
    }
    if (!state && !age)
        return FS_OK;
    void* tmp = nullptr;
    if (!g->identity)
        FS_CUDA(s, fs::dmalloc(&tmp, (size_t)n * 4));
    fs_status rc = FS_OK;
    auto copy_out = [&](const void* dsrc, void* hdst, int eb) -> cudaError_t {
        if (g->identity)
            return cudaMemcpy(hdst, dsrc, (size_t)n * eb, cudaMemcpyDeviceToHost);
        cudaError_t e = fs::launch_to_original(dsrc, tmp, eb, g->d_perm, n, s->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy(hdst, tmp, (size_t)n * eb, cudaMemcpyDeviceToHost);
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (state)
        e = copy_out(s->d_X, state, 1);
    if (e == cudaSuccess && age)
        e = copy_out(s->d_A, age, s->age_bytes);
    if (e != cudaSuccess) {
        s->failed = true;
        rc = fail(FS_ECUDA, "get_state: %s", cudaGetErrorString(e));
    }
    fs::dfree(tmp);
    return rc;
}

// storage value of an age: S and R ages must be +-0, E and I ages finite and >= 0
static bool age_ok(const void* age, int dtype, int64_t i, bool must_be_zero)
{
    if (dtype == FS_AGE_F32) {
        const float v = ((const float*)age)[i];
        return must_be_zero ? (v == 0.0f) : (std::isfinite(v) && v >= 0.0f);
    }
    const uint16_t b = ((const uint16_t*)age)[i];
    if ((b & 0x7fffu) == 0)
        return true;
    if (must_be_zero || (b & 0x8000u))
        return false;
    if (dtype == FS_AGE_F16)
        return ((b >> 10) & 0x1fu) != 0x1fu;
    return ((b >> 7) & 0xffu) != 0xffu;
}

fs_status fs_sim_set_state(fs_sim* s, const uint8_t* state, const void* age, int64_t step)
{
    if (!s || !state || !age)
        return fail(FS_EINVAL, "NULL argument");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    if (step < 0 || step >= ((int64_t)1 << 32))
        return fail(FS_EINVAL, "step must be in [0, 2^32)");
    const fs_graph* g = s->g;
    const int n = (int)g->n;
    for (int64_t i = 0; i < n; ++i) {
        const int x = state[i];
        if (x > FS_R || (s->p.model != FS_SEIR && x == FS_E) || (s->p.model == FS_SIS && x == FS_R))
            return fail(FS_EINVAL, "state[%lld] = %d is not a compartment of the model", (long long)i, x);
        if (!age_ok(age, s->p.age_dtype, i, x == FS_S || x == FS_R))
            return fail(FS_EINVAL, "age[%lld] invalid (S/R ages must be 0; E/I ages finite and >= 0)",
                        (long long)i);
    }
    FS_CUDA(s, cudaStreamSynchronize(s->stream));
    void* tmp = nullptr;
    if (!g->identity)
        FS_CUDA(s, fs::dmalloc(&tmp, (size_t)n * 4));
    cudaError_t e = cudaSuccess;
    auto copy_in = [&](const void* hsrc, void* ddst, int eb) -> cudaError_t {
        if (g->identity)
            return cudaMemcpy(ddst, hsrc, (size_t)n * eb, cudaMemcpyHostToDevice);
        cudaError_t e2 = cudaMemcpy(tmp, hsrc, (size_t)n * eb, cudaMemcpyHostToDevice);
        if (e2 == cudaSuccess)
            e2 = fs::launch_from_original(tmp, ddst, eb, g->d_inv, n, s->stream);
        if (e2 == cudaSuccess)
            e2 = cudaStreamSynchronize(s->stream);
        return e2;
    };
    e = copy_in(state, s->d_X, 1);
    if (e == cudaSuccess)
        e = copy_in(age, s->d_A, s->age_bytes);
    fs::dfree(tmp);
    if (e != cudaSuccess) {
        s->failed = true;
        return fail(FS_ECUDA, "set_state: %s", cudaGetErrorString(e));
    }
    fs::DevCtl c{};
    c.step = step;
    FS_CUDA(s, cudaMemcpy(s->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice));
    FS_CUDA(s, fs::launch_refresh(s->d_X, n, g->d_deg, s->d_bm[0], s->d_bm[1], s->d_ctl, s->stream));
    if (s->pressure == FS_PRESSURE_PUSH)
        FS_CUDA(s, push_reset(s));
    if (s->d_rho[0])
        FS_CUDA(s, fs::launch_rho_init(step_args(s, 0), s->p.age_dtype, (uint32_t)(step & 1), s->stream));
    if (s->markov)
        FS_CUDA(s, fs::launch_markov_recount(step_args(s, 0), s->stream, s->g->num_sms));
    FS_CUDA(s, cudaStreamSynchronize(s->stream));
    return FS_OK;
}

fs_status fs_sim_active_units(const fs_sim* s, uint64_t* listed, uint64_t* units)
{
    if (!s || !listed || !units)
        return fail(FS_EINVAL, "NULL argument");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    fs::DevCtl c;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(&c, s->d_ctl, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_sim_active_units: %s", cudaGetErrorString(e));
    *listed = c.act_sum;
    *units = 0;
    if (s->d_act)
        *units = s->pressure == FS_PRESSURE_PUSH
                     ? (uint64_t)(((int64_t)s->g->n_thr + fs::kPushG - 1) / fs::kPushG + s->g->n_m)
                     : (uint64_t)s->g->n_slices;
    return FS_OK;
}

fs_status fs_sim_transitions(const fs_sim* s, uint64_t* total)
{
    if (!s || !total)
        return fail(FS_EINVAL, "NULL argument");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    fs::DevCtl c;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(&c, s->d_ctl, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_sim_transitions: %s", cudaGetErrorString(e));
    *total = c.transitions;
    return FS_OK;
}

fs_status fs_sim_infectivity_get(fs_sim* s, void* rho)
{
    if (!s || !rho)
        return fail(FS_EINVAL, "NULL argument");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    if (!s->d_rho[0])
        return fail(FS_EUNSUPPORTED, "fs_sim_infectivity_get: the sim has no shedding profile");
    const int64_t n = s->g->n;
    std::vector<uint8_t> X((size_t)std::max<int64_t>(n, 1));
    int64_t step = 0;
    fs_status st = fs_sim_get_state(s, X.data(), nullptr, &step);
    if (st != FS_OK)
        return st;
    const fs_graph* g = s->g;
    const int eb = s->age_bytes;
    const void* src = s->d_rho[step & 1];
    cudaError_t e = cudaSuccess;
    if (g->identity) {
        e = cudaMemcpy(rho, src, (size_t)n * eb, cudaMemcpyDeviceToHost);
    } else {
        void* tmp = nullptr;
        e = fs::dmalloc(&tmp, (size_t)std::max<int64_t>(n, 1) * eb);
        if (e == cudaSuccess)
            e = fs::launch_to_original(src, tmp, eb, g->d_perm, (int)n, s->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy(rho, tmp, (size_t)n * eb, cudaMemcpyDeviceToHost);
        fs::dfree(tmp);
    }
    if (e != cudaSuccess) {
        s->failed = true;
        return fail(FS_ECUDA, "fs_sim_infectivity_get: %s", cudaGetErrorString(e));
    }
    // entries of non-I nodes are stale in the device buffer (never read)
    unsigned char* out = static_cast<unsigned char*>(rho);
    for (int64_t i = 0; i < n; ++i)
        if (X[(size_t)i] != FS_I)
            memset(out + (size_t)i * eb, 0, (size_t)eb);
    return FS_OK;
}

fs_status fs_sim_time(const fs_sim* s, double* elapsed, float* next_dt)
{
    if (!s)
        return fail(FS_EINVAL, "sim is NULL");
    if (s->failed)
        return fail(FS_ESTATE, "sim is in a failed state");
    fs::DevCtl c;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(&c, s->d_ctl, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_sim_time: %s", cudaGetErrorString(e));
    if (elapsed)
        *elapsed = c.time;
    if (next_dt) {
        float dt = s->markov ? 0.0f : s->M.dt;       // Markovian: known only from the state's rates
        if (s->d_dtrec && !s->markov) {
            // the device's own rule, in the same FP32 operations
            uint32_t bits = c.lam[(c.step + 2) % 3];
            float lp;
            memcpy(&lp, &bits, sizeof(lp));
            const float eps = (float)s->p.eps, delta = (float)(s->p.delta > 0 ? s->p.delta : 1e-12);
            const float q = eps / (lp + delta);
            dt = q < dt ? q : dt;
        }
        *next_dt = dt;
    }
    return FS_OK;
}

fs_status fs_sim_pressure_get(const fs_sim* s, int32_t* pressure)
{
    if (!s || !pressure)
        return fail(FS_EINVAL, "NULL argument");
    *pressure = s->pressure;
    return FS_OK;
}

fs_status fs_sim_work(const fs_sim* s, uint64_t* s_degree_sum, uint64_t* s_node_sum, int64_t* steps_run)
{
    if (!s)
        return fail(FS_EINVAL, "sim is NULL");
    fs::DevCtl c;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(&c, s->d_ctl, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_sim_work: %s", cudaGetErrorString(e));
    if (s_degree_sum)
        *s_degree_sum = c.ds_total;
    if (s_node_sum)
        *s_node_sum = c.s_total;
    if (steps_run)
        *steps_run = c.step;
    return FS_OK;
}

fs_status fs_sim_destroy(fs_sim* s)
{
    if (!s)
        return fail(FS_EINVAL, "sim is NULL");
    cudaStreamSynchronize(s->stream);
    s->g->refs -= 1;
    free_sim(s);
    return FS_OK;
}

fs_status fs_eval_hazard(const fs_law* law, const float* tau_dev, float* h_dev, int64_t n, void* stream)
{
    if (!law || n < 0 || (n > 0 && (!tau_dev || !h_dev)))
        return fail(FS_EINVAL, "bad argument");
    fs_status st = check_law(*law, "eval", false);
    if (st != FS_OK)
        return st;
    cudaError_t e = fs::launch_eval_hazard(to_lawf(*law), tau_dev, h_dev, n, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_eval_hazard: %s", cudaGetErrorString(e));
    return FS_OK;
}

fs_status fs_eval_density(const fs_law* law, const float* tau_dev, float* f_dev, int64_t n, void* stream)
{
    if (!law || n < 0 || (n > 0 && (!tau_dev || !f_dev)))
        return fail(FS_EINVAL, "bad argument");
    fs_status st = check_law(*law, "eval", false);
    if (st != FS_OK)
        return st;
    cudaError_t e = fs::launch_eval_density(to_lawf(*law), tau_dev, f_dev, n, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_eval_density: %s", cudaGetErrorString(e));
    return FS_OK;
}

fs_status fs_eval_uniforms(uint64_t seed, uint32_t replicate, int64_t step, const int32_t* nodes_dev, float* u_dev,
                           int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!nodes_dev || !u_dev)) || step < 0 || step >= ((int64_t)1 << 32))
        return fail(FS_EINVAL, "bad argument");
    cudaError_t e = fs::launch_eval_uniforms((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), replicate,
                                             (uint32_t)step, nodes_dev, u_dev, n, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_eval_uniforms: %s", cudaGetErrorString(e));
    return FS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// fs_step_noalloc: one fused step that allocates nothing. Its scratch (the
// merge class's cross-chunk partial counts and tickets, the control block the
// step kernel reads its step index from and writes its error word to, and the
// step's row of delta slots) lives in one file-scope device array, looked up
// once per device.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxMergeRows = 65536;
constexpr size_t kNoAllocCtlBytes = 256;
constexpr size_t kNoAllocSlotBytes = sizeof(unsigned long long) * fs::kDeltaRow;   // one step's delta slots
constexpr size_t kNoAllocBytes = kNoAllocCtlBytes + kNoAllocSlotBytes + (size_t)kNoAllocMaxMergeRows * 8;
static_assert(sizeof(fs::DevCtl) <= kNoAllocCtlBytes, "control block does not fit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (set-up on the
// first call per device; host code may not use the symbol's host stand-in)
fs_status noalloc_scratch_addr(unsigned char** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_step_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(FS_EUNSUPPORTED, "fs_step_noalloc: device ordinal %d beyond %d", dev, kNoAllocMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(FS_ECUDA, "fs_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    return FS_OK;
}

// clears the scratch rows in use and the delta slots, sets the step index
// (everything the step expects to start at zero)
__global__ void noalloc_prepare_kernel(fs::DevCtl* ctl, int32_t* cnt, uint32_t* tkt, int n_m, int64_t step,
                                       unsigned long long* slots)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = t; i < n_m; i += (int64_t)gridDim.x * blockDim.x) {
        cnt[i] = 0;
        tkt[i] = 0u;
    }
    if (t == 0) {
        ctl->step = step;
        ctl->error = 0;
    }
    if (t < fs::kDeltaRow)
        slots[t] = 0ull;
}

// the step's totals (the delta slots summed) and the device error word into
// the caller's five words; one warp, lane = slot
__global__ void noalloc_finish_kernel(const fs::DevCtl* ctl, const unsigned long long* slots,
                                      unsigned long long* deltas)
{
    static_assert(fs::kDeltaSlots == 32, "one delta slot per lane");
    const int lane = threadIdx.x & 31;
    unsigned long long f[fs::kDeltaFields];
    for (int q = 0; q < fs::kDeltaFields; ++q) {
        f[q] = slots[lane * fs::kDeltaFields + q];
        for (int o = 16; o > 0; o >>= 1)
            f[q] += __shfl_xor_sync(0xffffffffu, f[q], o);
    }
    if (lane == 0) {
        for (int q = 0; q < fs::kDeltaFields; ++q)
            deltas[q] = f[q];
        deltas[4] = (unsigned long long)(unsigned)ctl->error;
    }
}

}  // namespace

extern "C" fs_status fs_step_noalloc(const fs_graph* g, const fs_sim_params* params, int64_t step,
                                     uint8_t* state_dev, void* age_dev, const uint32_t* bitmap_cur_dev,
                                     uint32_t* bitmap_next_dev, uint64_t* deltas_dev, void* stream)
{
    g_err.clear();
    if (!g || !state_dev || !age_dev || !bitmap_cur_dev || !bitmap_next_dev || !deltas_dev)
        return fail(FS_EINVAL, "fs_step_noalloc: NULL argument");
    if (g->failed)
        return fail(FS_ESTATE, "fs_step_noalloc: graph is in a failed state");
    if (!params)
        return fail(FS_EINVAL, "fs_step_noalloc: params is NULL");
    fs_sim_params pv = *params;                     // index_state does not apply to one step
    pv.index_state = pv.model == FS_SEIR ? FS_E : FS_I;
    fs_status st = check_params(&pv);
    if (st != FS_OK)
        return st;
    if (pv.eps > 0)
        return fail(FS_EUNSUPPORTED, "fs_step_noalloc: one step has a fixed size (eps must be 0)");
    if (pv.shed_mode != FS_SHED_NONE)
        return fail(FS_EUNSUPPORTED, "fs_step_noalloc: a shedding profile needs the sim's infectivity buffers");
    if (pv.flags & FS_ACTIVE_LIST)
        return fail(FS_EUNSUPPORTED, "fs_step_noalloc: FS_ACTIVE_LIST needs the sim's launch sequences");
    if (pv.theta > 0)
        return fail(FS_EUNSUPPORTED, "fs_step_noalloc: the Markovian engine needs the sim's count buffers");
    if (step < 0 || step >= ((int64_t)1 << 32))
        return fail(FS_EINVAL, "fs_step_noalloc: step must be in [0, 2^32)");
    if (g->n_m > kNoAllocMaxMergeRows)
        return fail(FS_EINVAL,
                    "fs_step_noalloc: the graph has %d merge-class rows; the allocation-free step supports at "
                    "most %d (raise thread_max_deg when creating the graph, or use fs_sim_*)",
                    g->n_m, kNoAllocMaxMergeRows);
    unsigned char* base = nullptr;
    st = noalloc_scratch_addr(&base);
    if (st != FS_OK)
        return st;
    fs::DevCtl* ctl = reinterpret_cast<fs::DevCtl*>(base);
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(base + kNoAllocCtlBytes);
    int32_t* cnt = reinterpret_cast<int32_t*>(base + kNoAllocCtlBytes + kNoAllocSlotBytes);
    uint32_t* tkt = reinterpret_cast<uint32_t*>(base + kNoAllocCtlBytes + kNoAllocSlotBytes +
                                                (size_t)kNoAllocMaxMergeRows * 4);
    cudaStream_t cs = (cudaStream_t)stream;
    unsigned long long* deltas = reinterpret_cast<unsigned long long*>(deltas_dev);

    const int prep_blocks = std::max(1, std::min(64, (g->n_m + 255) / 256));
    noalloc_prepare_kernel<<<prep_blocks, 256, 0, cs>>>(ctl, cnt, tkt, g->n_m, step, slots);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_step_noalloc: prepare: %s", cudaGetErrorString(e));
    fs::g_launch_count += 1;

    fs::StepArgs a{};
    a.X = state_dev;
    a.A = age_dev;
    a.bm[step & 1] = const_cast<uint32_t*>(bitmap_cur_dev);
    a.bm[(step + 1) & 1] = bitmap_next_dev;
    a.sell_off = g->d_sell_off;
    a.sell_col = g->d_sell_col;
    a.n_thr = g->n_thr;
    a.n_slices = g->n_slices;
    a.sentinel = (int32_t)g->n;
    a.m_base = g->n_thr;
    a.n_m = g->n_m;
    a.n_chunks = g->n_chunks;
    a.spw = g->spw;
    a.n_sell_ctas = (g->n_slices + fs::kSellSlicesPerCta * g->spw - 1) / (fs::kSellSlicesPerCta * g->spw);
    a.m_ptr = g->d_m_ptr;
    a.m_col = g->d_m_col;
    a.m_warp_row = g->d_m_warp_row;
    a.m_chunk_last = g->d_m_chunk_last;
    a.e_m = g->e_m;
    a.m_cnt = cnt;
    a.m_tkt = tkt;
    a.perm = g->d_perm;
    a.deg = g->d_deg;
    a.M = to_model(pv);
    a.ctl = ctl;
    a.deltas = slots;
    a.j = 0;
    a.n = (int32_t)g->n;
    e = fs::launch_step(a, pv.age_dtype, cs, false);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_step_noalloc: step: %s", cudaGetErrorString(e));
    noalloc_finish_kernel<<<1, 32, 0, cs>>>(ctl, slots, deltas);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(FS_ECUDA, "fs_step_noalloc: finish: %s", cudaGetErrorString(e));
    fs::g_launch_count += 1;
    return FS_OK;
}
