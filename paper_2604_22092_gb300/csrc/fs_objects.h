// fs_objects.h -- host-side definitions of the opaque handles of include/fs.h
// (internal to libflashstep; shared by the C-ABI translation units).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "fs.h"
#include "fs_internal.h"

namespace fs {
// device memory of the library (fs_alloc.cpp): freed blocks are cached by
// size and handed out again, or every block comes from the caller's
// allocator (fs_set_allocator)
cudaError_t dmalloc_raw(void** p, size_t bytes);
cudaError_t dfree(void* p);
template <class T>
inline cudaError_t dmalloc(T** p, size_t bytes)
{
    return dmalloc_raw(reinterpret_cast<void**>(p), bytes);
}
}  // namespace fs

struct fs_graph {
    int64_t n = 0, nnz = 0;
    int32_t dmax = 0;
    int32_t t1 = 0;
    int32_t n_thr = 0, n_m = 0, n_slices = 0, n_chunks = 0;
    int64_t e_m = 0, sell_entries = 0;
    bool identity = true;
    int32_t* d_perm = nullptr;     // internal -> original
    int32_t* d_inv = nullptr;      // original -> internal
    int32_t* d_deg = nullptr;      // degree by internal id
    int64_t* d_sell_off = nullptr;
    int32_t* d_sell_col = nullptr;
    int64_t* d_m_ptr = nullptr;
    int32_t* d_m_col = nullptr;
    int32_t* d_m_warp_row = nullptr;
    int32_t* d_m_chunk_last = nullptr;
    int64_t bytes = 0;
    int32_t num_sms = 152;
    int32_t spw = 1;               // SELL slices per warp (one wave of step CTAs)
    uint32_t bm_bytes = 0;         // infectious bitmap bytes, rounded up to 16
    bool smem_path = false;        // bitmap small enough to be staged in shared memory
    uint32_t smem_min_s = 0;       // S count from which staging pays off
    // transposed CSR (internal ids) for the push form of the pressure, built
    // on the first push-form sim of the graph
    int64_t* d_out_ptr = nullptr;  // [n + 1]
    int32_t* d_out_col = nullptr;  // [nnz], inside the allocation of d_out_ptr
    int refs = 0;
    bool failed = false;
};

struct fs_sim {
    fs_graph* g = nullptr;
    void* d_arena = nullptr;       // one allocation holding every per-sim device buffer below
    fs_sim_params p{};
    fs::ModelF M{};
    int age_bytes = 4;
    uint8_t* d_X = nullptr;
    void* d_A = nullptr;
    uint32_t* d_bm[2] = {nullptr, nullptr};
    int32_t* d_m_cnt = nullptr;
    uint32_t* d_m_tkt = nullptr;
    fs::DevCtl* d_ctl = nullptr;
    unsigned long long* d_deltas = nullptr;
    float4* d_ptab = nullptr;
    float* d_ps = nullptr;
    // adaptive step (p.eps > 0): the step sizes of the current launch sequence
    float* d_dtrec = nullptr;
    // shedding profile (p.shed_mode != 0): infectivity by step parity, and
    // the merge class's cross-chunk partial pressures
    void* d_rho[2] = {nullptr, nullptr};
    float2* d_mpart = nullptr;
    float4* d_rtab = nullptr;     // [kPTableN] memoised beta s(age)
    int32_t* d_act = nullptr;     // active-node compaction list (FS_ACTIVE_LIST)
    // Markovian engine (p.theta > 0): exact counts and the step's event list
    bool markov = false;
    uint32_t* d_mk_cnt = nullptr;
    uint32_t* d_mk_ev = nullptr;
    // push form of the pressure (pressure == FS_PRESSURE_PUSH)
    int pressure = FS_PRESSURE_GATHER;
    uint8_t* d_cnt8 = nullptr;
    uint16_t* d_pd16[2] = {nullptr, nullptr};
    uint32_t* d_hcnt = nullptr;
    unsigned long long* d_pd64[2] = {nullptr, nullptr};
    uint32_t* d_counts = nullptr;
    int64_t counts_cap = 0;
    cudaGraphExec_t gexec = nullptr;
    int gK = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool failed = false;
    // failure-detection test settings in force when the sim was created
    // (fs_test_inject): wait limit with no bulk copies, bounds-check shrink
    uint32_t test_wait_limit = 0;
    int64_t test_bounds_shrink = 0;
};


// helpers of the C-ABI translation units (fs_api.cu)
namespace fsapi {
extern thread_local std::string g_err;
fs_status fail(fs_status st, const char* fmt, ...);
// cudaMalloc of count elements (at least one), adding the bytes to *bytes
template <typename T>
inline cudaError_t dev_alloc(T** p, size_t count, int64_t* bytes)
{
    const size_t b = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = fs::dmalloc((void**)p, b);
    if (e == cudaSuccess && bytes)
        *bytes += (int64_t)b;
    return e;
}
// scratch of the ingest (freed before fs_graph_create / fs_sim_init return)
template <typename T>
inline cudaError_t scratch_alloc(T** p, size_t count, cudaStream_t)
{
    return fs::dmalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
}
inline void scratch_free(void* p, cudaStream_t)
{
    fs::dfree(p);
}
fs_status check_params(const fs_sim_params* p);
fs::ModelF to_model(const fs_sim_params& p);
fs::LawF to_lawf(const fs_law& L);
// the push form of the pressure: available when the thread class's in-degrees
// fit u8 counts; the transposed CSR of a graph, built once (thread-safe)
bool push_available(const fs_graph* g);
// the pressure form of a packed ensemble of n_real realisations (fs_pack_api.cu)
bool packed_push(const fs_graph* g, const fs_sim_params& p0, int n_real);
cudaError_t ensure_out_csr(fs_graph* g, cudaStream_t st);
// the dispatch autotuner (fs_tune.cpp): builds the graph with the class split
// it chooses for this degree profile (base: the caller's options, AUTO)
fs_status tune_create(int64_t n, int64_t nnz, int64_t dmax, const int64_t* row_ptr, const int32_t* col_ind,
                      const fs_graph_opts& base, void* stream, fs_graph** out);

}  // namespace fsapi
