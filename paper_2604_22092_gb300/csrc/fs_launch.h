// fs_launch.h -- host-side launchers of the kernels in fs_step.cu and
// fs_ingest.cu (internal to libflashstep).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "fs_internal.h"

namespace fs {

// kernels enqueued by this library (graph replays add their node count)
extern std::atomic<unsigned long long> g_launch_count;

// fs_step.cu
// pdl: launch with programmatic stream serialization (overlaps the launch
// with the previous kernel; the kernel waits for it before reading anything)
cudaError_t launch_step(const StepArgs& a, int age_dtype, cudaStream_t s, bool pdl);
// one step as the shared-memory-bitmap SELL grid plus, if present, the merge grid
cudaError_t launch_step_smem(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms);
// rtab (optional): the memoised infectivity beta s(age) of a shedding profile
cudaError_t launch_build_ptables(const ModelF& M, int age_dtype, float4* tab, float* ps, cudaStream_t s,
                                 float4* rtab = nullptr, const LawF& shed = LawF{}, int shed_mode = 0);
cudaError_t launch_run_begin(DevCtl* ctl, uint32_t* out, cudaStream_t s);
// dtrec: the K step sizes (adaptive step) or null (every step is dt)
cudaError_t launch_run_epilogue(DevCtl* ctl, unsigned long long* deltas, int K, int model, const float* dtrec,
                                float dt, cudaStream_t s);
// one step of the push form with the adaptive step
cudaError_t launch_push_step_adaptive(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms);
cudaError_t launch_refresh(const uint8_t* X, int n, const int32_t* deg, uint32_t* bm0, uint32_t* bm1, DevCtl* ctl,
                           cudaStream_t s);
cudaError_t launch_set_index(uint8_t* X, const int32_t* idx, int64_t n_idx, const int32_t* inv, int state,
                             cudaStream_t s);
cudaError_t launch_to_original(const void* in, void* out, int elem_bytes, const int32_t* perm, int n, cudaStream_t s);
cudaError_t launch_from_original(const void* in, void* out, int elem_bytes, const int32_t* inv, int n,
                                 cudaStream_t s);
cudaError_t launch_eval_hazard(const LawF& L, const float* tau, float* h, int64_t n, cudaStream_t s);
cudaError_t launch_eval_density(const LawF& L, const float* tau, float* f, int64_t n, cudaStream_t s);
// Markovian engine: one step of Algorithm 1 (three launches), and the dense
// recount of the counts (after init or set_state)
cudaError_t launch_markov_step(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms);
cudaError_t launch_markov_recount(const StepArgs& a, cudaStream_t s, int num_sms);
// active-node compaction refreshes (a.act must be set): gather form (SELL
// slices) and push form (push items)
cudaError_t launch_sell_compact(const StepArgs& a, cudaStream_t s, int num_sms);
cudaError_t launch_push_compact(const StepArgs& a, cudaStream_t s, int num_sms);
// rho[par] of every I node from its age (a.X, a.A, a.rho, a.M.beta, a.shed*)
cudaError_t launch_rho_init(const StepArgs& a, int age_dtype, uint32_t par, cudaStream_t s);
cudaError_t launch_eval_uniforms(uint32_t key0, uint32_t key1, uint32_t rep, uint32_t step, const int32_t* nodes,
                                 float* u, int64_t n, cudaStream_t s);

// fs_push.cu: one step with the pressure kept by pushes; the initial counts
// (counts and pending tallies zeroed before); the transposed CSR of a graph
// (fill = false: out-degrees into cursor; fill = true: rows via cursor)
cudaError_t launch_push_step(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms);
cudaError_t launch_push_init(const StepArgs& a, cudaStream_t s, int num_sms);
cudaError_t launch_transpose(const int64_t* sell_off, const int32_t* sell_col, const int32_t* deg, int n_thr,
                             const int64_t* m_ptr, const int32_t* m_col, int n_m, int n,
                             unsigned long long* cursor, int32_t* out_col, bool fill, cudaStream_t s);

// fs_pack.cu
// one step of the segments of replicate-width class cls (R_pad = 8 << cls) in
// one pressure form (0 gather, 1 push, 2 gather with a shedding profile)
cudaError_t launch_pack_step(const PackArgs& a, int cls, int form, bool adaptive, int age_dtype, int grid,
                             cudaStream_t s);
cudaError_t launch_pack_init(uint8_t* X, int n, int R_pad, int R, const int32_t* idx, int64_t n_idx,
                             const int32_t* inv, int state, void* mask, cudaStream_t s);
int pack_grid(int num_sms, int cls);   // persistent grid of the packed step kernel of class cls
// initial counts of a push-form segment from its state (counts zeroed before)
cudaError_t launch_pack_push_init(const PackSeg& g, cudaStream_t s);
// rho[par] of the replicates that start in I (shedding profile)
cudaError_t launch_pack_rho_init(const PackSeg& g, int age_dtype, uint32_t par, cudaStream_t s);
cudaError_t launch_pack_advance(DevCtl* ctl, int K, cudaStream_t s);   // global step += K

// fs_ingest.cu
struct IngestFlags {
    int32_t dmax;
    int32_t unsorted;     // 1 when the class keys are not nondecreasing
    int32_t error;        // 1 = bad row_ptr, 2 = col_ind out of range
    int32_t n_thr;        // nodes with degree <= thread_max_deg
};
cudaError_t launch_degrees(const int64_t* row_ptr, int n, int t1, int32_t* deg, uint16_t* key, IngestFlags* flags,
                           cudaStream_t s);
cudaError_t launch_check_cols(const int32_t* col, int64_t nnz, int n, IngestFlags* flags, cudaStream_t s);
// stable counting sort of nodes by key (keys < n_buckets): perm[pos] = i, inv[i] = pos, deg_int[pos] = deg[i]
cudaError_t stable_sort_by_key(const uint16_t* key, const int32_t* deg, int n, int n_buckets, int32_t* perm,
                               int32_t* inv, int32_t* deg_int, cudaStream_t s);
// out[0..n] = exclusive prefix sums of in[0..n-1] (out[n] = total)
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
cudaError_t launch_sell_widths(const int32_t* deg_int, int n_thr, int n_slices, int64_t* width32, cudaStream_t s);
cudaError_t launch_sell_fill(const int64_t* row_ptr, const int32_t* col, const int32_t* perm, const int32_t* inv,
                             const int32_t* deg_int, int n_thr, int n_slices, const int64_t* sell_off, int sentinel,
                             int32_t* sell_col, cudaStream_t s);
cudaError_t launch_merge_degrees(const int32_t* deg_int, int m_base, int n_m, int64_t* out, cudaStream_t s);
cudaError_t launch_merge_fill(const int64_t* row_ptr, const int32_t* col, const int32_t* perm, const int32_t* inv,
                              int m_base, int n_m, const int64_t* m_ptr, int64_t e_m, int64_t padded, int sentinel,
                              int32_t* m_col, cudaStream_t s);
cudaError_t launch_merge_tables(const int64_t* m_ptr, int n_m, int64_t e_m, int n_chunks, int32_t* warp_row,
                                int32_t* chunk_last, cudaStream_t s);

}  // namespace fs
