// fs_step.cu -- the fused renewal tau-leaping step (FlashSpread, arXiv
// 2604.22092, Algorithm 3 at a fixed step) for one realisation, plus the
// small kernels around it (run begin/epilogue, state refresh, relabelling,
// diagnostics).
//
// One launch performs one whole step for every node. The grid has two kinds
// of CTA (Section 5.5, degree-aware traversal):
//   * merge CTAs (blockIdx < n_chunks): one 4096-edge chunk of the merge
//     class (rows of degree > thread_max_deg). The chunk's column block is
//     staged in shared memory by one bulk TMA copy; each warp counts the
//     infectious in-neighbours of the rows overlapping its 512 edges with
//     ballots over 32-edge windows; rows that span chunks combine integer
//     partial counts with an atomic ticket (the last chunk runs the tail), so
//     the result is exact and independent of scheduling.
//   * SELL CTAs: eight 32-node slices of the one-thread-per-node class stored
//     as SELL-32 (column-major 32-wide blocks), one lane per node.
// Only S nodes read their row; the neighbour infectivity is a 1-bit
// infectious bitmap (Eq. 8 with s = 1), read through the read-only path and
// double-buffered by step parity; the next bitmap is written with warp
// ballots. States and ages are updated in place (each node has one owner).
#include <cuda_runtime.h>

#include <algorithm>

#include "fs_device.cuh"
#include "fs_launch.h"

namespace fs {

std::atomic<unsigned long long> g_launch_count{0};

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ void record_error(DevCtl* ctl, int code)
{
    atomicCAS(&ctl->error, 0, code);
}

__device__ __forceinline__ uint32_t orig_id(const int32_t* perm, int i)
{
    return perm ? (uint32_t)__ldg(perm + i) : (uint32_t)i;
}

// direct evaluation (rare path: ages off the tabulated sequence); kept out of
// line so that its registers do not weigh on the common path
__device__ __noinline__ float p_direct(const ModelF& M, int x, float age)
{
    return p_of_rate(M, hazard(x == kE ? M.lat : M.inf, age));
}

// Bernoulli probability of one node this step (Section 5.2): S nodes from
// beta * c, E/I nodes from the hazard at their begin-of-step age. Both come
// from per-sim tables built by the same FP32 code at init (identical bits);
// ages off the fixed-step sequence, counts beyond the S table, and launches
// without tables (null pointers) are evaluated directly.
__device__ __forceinline__ float node_p(const StepArgs& a, int x, float age, uint32_t c)
{
    if (x == kS) {
        if (c == 0u)
            return 0.0f;
        if (a.ps && c < (uint32_t)kPSTableN)
            return __ldg(a.ps + c);
        return p_of_rate(a.M, __fmul_rn(a.M.beta, (float)c));
    }
    if (x == kE || x == kI) {
        const int n = __float2int_rn(__fmul_rn(age, a.M.inv_dt));
        if (a.ptab && (unsigned)n < (unsigned)kPTableN) {
            const float4* row = a.ptab + (x == kI ? kPTableN : 0) + n;
            const float2 e = __ldg(reinterpret_cast<const float2*>(row));
            if (e.x == age)
                return e.y;
            const float p1 = ptab_slot1(row, age);
            if (p1 >= 0.0f)
                return p1;
        }
        return p_direct(a.M, x, age);
    }
    return 0.0f;
}

// beta s(tau) of an I node of age tau (Eq. 8), FP32; out of line (I nodes
// only, and only in the SHED instances)
__device__ __noinline__ float shed_rho(const StepArgs& a, float tau)
{
    return shed_value(a.shed, a.shed_mode, a.M.beta, tau);
}

// the same value from the per-sim table when the age is on the fixed-step
// sequence (identical bits: the table is built by shed_value)
__device__ __forceinline__ float rho_of_age(const StepArgs& a, float age)
{
    const int n = __float2int_rn(__fmul_rn(age, a.M.inv_dt));
    if ((unsigned)n < (unsigned)kPTableN) {
        const float4* row = a.rtab + n;
        const float2 e = __ldg(reinterpret_cast<const float2*>(row));
        if (e.x == age)
            return e.y;
        const float r1 = ptab_slot1(row, age);
        if (r1 >= 0.0f)
            return r1;
    }
    return shed_rho(a, age);
}

// Bernoulli decision and transition for one node of probability p
// (Algorithm 3); the original id is looked up only when a uniform is needed
__device__ __forceinline__ TailResult tail_p_dt(const StepArgs& a, int x, float age, float p, int i, uint32_t step,
                                                float dt)
{
    bool fired = false;
    if (p > 0.0f)
        fired = uniform24(a.M.key0, a.M.key1, a.M.rep, step, orig_id(a.perm, i)) < p;
    TailResult r;
    if (fired) {
        r.x = (x == kS) ? (a.M.model == kSEIR ? kE : kI) : (x + 1);
        r.age = 0.0f;
    } else {
        r.x = x;
        r.age = (x == kE || x == kI) ? __fadd_rn(age, dt) : 0.0f;
    }
    r.fired = fired;
    return r;
}

__device__ __forceinline__ TailResult tail_p(const StepArgs& a, int x, float age, float p, int i, uint32_t step)
{
    return tail_p_dt(a, x, age, p, i, step, a.M.dt);
}

// the E / I rate evaluated directly (adaptive step: ages leave the fixed-step
// sequence of the tables); out of line
__device__ __noinline__ float hazard_of(const ModelF& M, int x, float age)
{
    return hazard(x == kE ? M.lat : M.inf, age);
}

// The variant bits of the gather kernels: kModeShed (source-node
// infectivity with a shedding profile, Eq. 8) and kModeAdaptive (the step
// size of Section 5.2 with rates evaluated directly).
constexpr int kModeShed = 1, kModeAdaptive = 2;

// the adaptive step's size for step k (every thread computes it); the first
// thread of the grid clears the rate slot read two steps ago and records it
__device__ __forceinline__ float adaptive_dt(const StepArgs& a, int64_t k)
{
    const float lp = __uint_as_float(a.ctl->lam[(k + 2) % 3]);
    const float dt = fminf(a.M.dt, __fdiv_rn(a.eps, __fadd_rn(lp, a.delta)));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->lam[(k + 1) % 3] = 0u;
        a.dtrec[a.j] = dt;
    }
    return dt;
}

// this thread's largest rate into the step's slot (rates are >= 0, so their
// FP32 bits order as unsigned integers); every lane of the warp calls it
__device__ __forceinline__ void adaptive_lmax(const StepArgs& a, int64_t k, float lmax)
{
    const uint32_t m = __reduce_max_sync(kFull, __float_as_uint(lmax));
    if ((threadIdx.x & 31) == 0 && m)
        atomicMax(&a.ctl->lam[k % 3], m);
}

__device__ __forceinline__ TailResult tail_at(const StepArgs& a, int x, float age, uint32_t c, int i,
                                              uint32_t step)
{
    return tail_p(a, x, age, node_p(a, x, age, c), i, step);
}

// ---------------------------------------------------------------------------
// One-thread-per-node class: a warp owns `spw` consecutive 32-node SELL
// slices; the states of four slices are loaded together so that their
// latencies overlap, then each slice is processed with one lane per node.
// ---------------------------------------------------------------------------
struct LaneDeltas {
    uint32_t fS = 0, fE = 0, fI = 0, dS = 0;
    float lmax = 0.0f;           // adaptive step: the largest rate this lane saw
};

template <typename AgeT, bool SMEM_BM, int MODE = 0>
__device__ __forceinline__ void sell_slice(const StepArgs& a, uint32_t step, const uint32_t* __restrict__ bm,
                                           uint32_t* __restrict__ bmn, int slice, int x, LaneDeltas& ld,
                                           float dt, uint32_t mbar = 0u, bool* ready = nullptr)
{
    constexpr bool SHED = (MODE & kModeShed) != 0, ADPT = (MODE & kModeAdaptive) != 0;
    constexpr int B = 12;                        // column loads in flight per lane
    const int lane = threadIdx.x & 31;
    const int i = slice * 32 + lane;
    const bool valid = i < a.n_thr;
    AgeT* __restrict__ A = static_cast<AgeT*>(a.A);
    float age = 0.0f;
    if (x == kE || x == kI)
        age = AgeIO<AgeT>::load(A[i]);
    uint32_t c = 0;
    float rs = 0.0f;                             // SHED: FP32 sum of the stored rho, row order
    if (x == kS) {
        // padding entries hold the sentinel id n, whose bitmap bit is always
        // 0, so every gathered bit is added without a test
        const int64_t off = __ldg(a.sell_off + slice);
        const int w = (int)((__ldg(a.sell_off + slice + 1) - off) >> 5);
        const int32_t* __restrict__ p = a.sell_col + off + lane;
        const int sentinel = a.sentinel;
        for (int t0 = 0; t0 < w; t0 += B) {
            int32_t jj[B];
#pragma unroll
            for (int u = 0; u < B; ++u)
                jj[u] = (t0 + u < w && FS_IN_BOUNDS(a.ctl, kSiteSellCol, off + lane + 32 * (int64_t)(t0 + u), a.sell_len))
                            ? __ldg(p + 32 * (t0 + u))
                            : sentinel;
            if constexpr (SMEM_BM) {
                // the shared copy of the bitmap is awaited only now, after
                // this lane's first column loads are in flight
                if (!*ready) {
                    if (!mbar_wait(mbar, 0u, a.wait_limit ? a.wait_limit : kWaitLimit))
                        record_error(a.ctl, kErrTmaTimeout);
                    *ready = true;
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                uint32_t word = 0u;
                if (!FS_IN_BOUNDS(a.ctl, kSiteBitmap, jj[u] >> 5, a.bm_words))
                    ;
                else if constexpr (SMEM_BM)
                    word = bm[jj[u] >> 5];
                else
                    word = __ldg(bm + (jj[u] >> 5));
                const uint32_t bit = __funnelshift_r(word, 0u, (uint32_t)jj[u]) & 1u;   // bit jj mod 32
                if constexpr (SHED) {
                    if (bit)
                        rs = __fadd_rn(rs, AgeIO<AgeT>::load(static_cast<const AgeT*>(a.rho[step & 1u])[jj[u]]));
                } else {
                    c += bit;
                }
            }
        }
    }
    TailResult r;
    if constexpr (ADPT) {
        float lam = 0.0f;
        if (x == kS)
            lam = SHED ? rs : (c ? __fmul_rn(a.M.beta, (float)c) : 0.0f);
        else if (x == kE || x == kI)
            lam = hazard_of(a.M, x, age);
        ld.lmax = fmaxf(ld.lmax, lam);
        r = tail_p_dt(a, x, age, p_of_rate_dt(lam, dt), i, step, dt);
    } else if constexpr (SHED) {
        r = tail_p(a, x, age, x == kS ? p_of_rate(a.M, rs) : node_p(a, x, age, 0u), i, step);
    } else {
        r = tail_at(a, x, age, c, i, step);
    }
    if (valid) {
        if (r.x != x)
            a.X[i] = (uint8_t)r.x;
        if (r.fired || x == kE || x == kI)
            A[i] = AgeIO<AgeT>::store(r.age);
        if constexpr (SHED) {
            if (r.x == kI)   // the next step's infectivity, from the new age as stored
                static_cast<AgeT*>(a.rho[(step & 1u) ^ 1u])[i] =
                    AgeIO<AgeT>::store(rho_of_age(a, AgeIO<AgeT>::load(AgeIO<AgeT>::store(r.age))));
        }
    }
    const uint32_t word = __ballot_sync(kFull, valid && r.x == kI);
    if ((slice + 1) * 32 <= a.n_thr) {
        if (lane == 0)
            bmn[slice] = word;
    } else {
        // the last slice shares its word with merge-class nodes: own bits only
        const uint32_t vmask = __ballot_sync(kFull, valid);
        if (lane == 0) {
            if (word)
                atomicOr(bmn + slice, word);
            atomicAnd(bmn + slice, word | ~vmask);
        }
    }
    if (r.fired) {
        ld.fS += x == kS;
        ld.fE += x == kE;
        ld.fI += x == kI;
        if (x == kS)
            ld.dS += (uint32_t)__ldg(a.deg + i);
    }
}

// Active-node compaction (Section 5.6): the SELL slices a step visits. With
// a list (ctl->n_act < n_slices), position q < n_act is the listed slice
// act[q]; without, position q is slice q. Positions past the end map to
// n_slices.
struct SliceMap {
    const int32_t* act;
    int n_items;
    bool list;
    // LIST is the run-time `list`, made a compile-time choice by the callers
    // so that the path without a list keeps its own register allocation
    template <bool LIST>
    __device__ __forceinline__ int at(int q) const
    {
        if constexpr (!LIST)
            return q;
        else
            return q < n_items ? __ldg(act + q) : INT32_MAX;
    }
};

__device__ __forceinline__ SliceMap slice_map(const StepArgs& a)
{
    SliceMap m{a.act, a.n_slices, false};
    if (a.act) {
        const unsigned long long na = a.ctl->n_act;
        if (na < (unsigned long long)a.n_slices) {
            m.list = true;
            m.n_items = (int)na;
        }
    }
    return m;
}

template <typename AgeT, int MODE, bool LIST>
__device__ __forceinline__ void sell_warp(const StepArgs& a, uint32_t step, const uint32_t* __restrict__ bm,
                                          uint32_t* __restrict__ bmn, int s_begin, int s_end, LaneDeltas& ld,
                                          const SliceMap& sm, float dt)
{
    const int lane = threadIdx.x & 31;
    for (int s0 = s_begin; s0 < s_end; s0 += 4) {
        uint32_t xs = 0;                       // four states, one byte each
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int sl = s0 + u < s_end ? sm.at<LIST>(s0 + u) : INT32_MAX;
            const uint32_t x = (sl < a.n_slices && sl * 32 + lane < a.n_thr) ? (uint32_t)a.X[sl * 32 + lane]
                                                                           : (uint32_t)kR;
            xs |= x << (8 * u);
        }
#pragma unroll 1
        for (int u = 0; u < 4; ++u) {
            if (s0 + u >= s_end)
                break;
            const int slice = sm.at<LIST>(s0 + u);
            if (slice >= a.n_slices)
                break;
            const int x = (int)((xs >> (8 * u)) & 0xffu);
            // absorbed slice: every node R, next-bitmap word 0, nothing else to do
            if (__all_sync(kFull, x == kR) && (slice + 1) * 32 <= a.n_thr) {
                if (lane == 0)
                    bmn[slice] = 0u;
                continue;
            }
            sell_slice<AgeT, false, MODE>(a, step, bm, bmn, slice, x, ld, dt);
        }
    }
}

// ---------------------------------------------------------------------------
// Merge class: one 4096-edge chunk per CTA.
// ---------------------------------------------------------------------------
struct MergeSmem {
    int32_t col[kMergeEPB];                 // staged column block (TMA destination)
    int64_t rp[kMergeMaxRows + 1];          // row bounds of the rows touched
    int32_t xs[kMergeMaxRows];              // their compartments
    uint32_t cnt[kMergeMaxRows];            // chunk-local infectious counts
    uint32_t wset[8], wclr[8];              // bitmap bits to set / clear
    unsigned long long mbar;
};

// SHED: per-warp partial pressures of the rows of its 32 lanes, and the
// first row of each warp's range (INT32_MAX: the warp has no edges)
template <bool SHED> struct MergeShedSmem {
    float part[kStepWarps][kWarp];
    int32_t wrow[kStepWarps];
};
template <> struct MergeShedSmem<false> {};

template <typename AgeT, int MODE>
__device__ __forceinline__ void merge_chunk(const StepArgs& a, uint32_t step, const uint32_t* __restrict__ bm,
                                            uint32_t* __restrict__ bmn, int chunk,
                                            float dt, float& lmax)
{
    constexpr bool SHED = (MODE & kModeShed) != 0, ADPT = (MODE & kModeAdaptive) != 0;
    __shared__ __align__(128) MergeSmem sm;
    __shared__ MergeShedSmem<SHED> sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e0 = (int64_t)chunk * kMergeEPB;
    const int64_t e1 = min(e0 + (int64_t)kMergeEPB, a.e_m);
    const int R0 = __ldg(a.m_warp_row + (int64_t)chunk * kStepWarps);
    const int R1 = __ldg(a.m_chunk_last + chunk);
    const int nrows = R1 - R0 + 1;           // <= kMergeMaxRows by construction
    AgeT* __restrict__ A = static_cast<AgeT*>(a.A);

    for (int t = tid; t <= nrows; t += kStepThreads)
        sm.rp[t] = __ldg(a.m_ptr + R0 + t);
    if (tid < 8) {
        sm.wset[tid] = 0u;
        sm.wclr[tid] = 0u;
    }
    int xrow = kR;
    if (tid < nrows) {
        xrow = a.X[a.m_base + R0 + tid];
        sm.xs[tid] = xrow;
        sm.cnt[tid] = 0u;
    }
    const int anyS = __syncthreads_or(xrow == kS);

    if (anyS) {
        const uint32_t mbar = smem_addr(&sm.mbar);
        const uint32_t bytes = kMergeEPB * 4u;
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                         : "memory");
            // (a failure-detection test sets skip_bulk_copy: the barrier then
            // waits for bytes that never come, with no copy in flight)
            if (!a.skip_bulk_copy)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_addr(sm.col)),
                    "l"(a.m_col + e0), "r"(bytes), "r"(mbar)
                    : "memory");
        }
        __syncthreads();
        const uint32_t lim = a.wait_limit ? a.wait_limit : kWaitLimit;
        bool ok = mbar_wait(mbar, 0u, lim);
        if (!ok) {
            record_error(a.ctl, kErrTmaTimeout);
            ok = mbar_wait(mbar, 0u, lim);          // let an in-flight copy land before leaving
        }
        const int64_t s0 = e0 + (int64_t)warp * kMergeEdgesPerWarp;
        if constexpr (SHED) {
            sh.part[warp][lane] = 0.0f;
            if (lane == 0)
                sh.wrow[warp] = INT32_MAX;
        }
        if (ok && s0 < e1) {
            const int64_t s1 = min(s0 + (int64_t)kMergeEdgesPerWarp, e1);
            const int rw = __ldg(a.m_warp_row + (int64_t)chunk * kStepWarps + warp);
            const int r = rw + lane;
            int64_t lo = 0, hi = 0;
            bool isS = false;
            if (r <= R1) {
                lo = max(sm.rp[r - R0], s0);
                hi = min(sm.rp[r - R0 + 1], s1);
                isS = sm.xs[r - R0] == kS;
            }
            const int32_t* cb = sm.col + (s0 - e0);
            if constexpr (SHED) {
                // each 32-edge window: lanes load the stored rho of their
                // edge's column if it is infectious and its row is S; a
                // segmented inclusive scan (fixed tree order) sums each row's
                // run of lanes; the row's lane adds the run's total, window
                // by window
                const AgeT* __restrict__ rho = static_cast<const AgeT*>(a.rho[step & 1u]);
                if (lane == 0)
                    sh.wrow[warp] = rw;
                float acc = 0.0f;
#pragma unroll 4
                for (int m = 0; m < kMergeWindowsPerWarp; ++m) {
                    const int64_t base = s0 + 32 * m;
                    const int l0 = (int)max((int64_t)0, min((int64_t)32, lo - base));
                    const int h0 = (int)max((int64_t)0, min((int64_t)32, hi - base));
                    uint32_t rm = 0u;
                    if (h0 > l0)
                        rm = ((h0 == 32) ? kFull : ((1u << h0) - 1u)) & ~((1u << l0) - 1u);
                    const uint32_t act = __reduce_or_sync(kFull, isS ? rm : 0u);
                    const uint32_t heads = __reduce_or_sync(kFull, h0 > l0 ? (1u << l0) : 0u);
                    float v = 0.0f;
                    if ((act >> lane) & 1u) {
                        const int32_t col = cb[32 * m + lane];
                        if ((__ldg(bm + (col >> 5)) >> (col & 31)) & 1u)
                            v = AgeIO<AgeT>::load(rho[col]);
                    }
                    const uint32_t below = heads & ((lane == 31) ? kFull : ((2u << lane) - 1u));
                    const int head = below ? 31 - __clz(below) : 0;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const float t = __shfl_up_sync(kFull, v, d);
                        if (lane - d >= head)
                            v = __fadd_rn(v, t);
                    }
                    const float seg = __shfl_sync(kFull, v, h0 > l0 ? h0 - 1 : 0);
                    if (isS && h0 > l0)
                        acc = __fadd_rn(acc, seg);
                }
                sh.part[warp][lane] = acc;
            } else {
            uint32_t cnt = 0;
#pragma unroll
            for (int m = 0; m < kMergeWindowsPerWarp; ++m) {
                const int64_t base = s0 + 32 * m;
                const int l0 = (int)max((int64_t)0, min((int64_t)32, lo - base));
                const int h0 = (int)max((int64_t)0, min((int64_t)32, hi - base));
                uint32_t rm = 0u;
                if (h0 > l0)
                    rm = ((h0 == 32) ? kFull : ((1u << h0) - 1u)) & ~((1u << l0) - 1u);
                const uint32_t act = __reduce_or_sync(kFull, isS ? rm : 0u);
                uint32_t bit = 0u;
                if ((act >> lane) & 1u) {
                    const int32_t col = cb[32 * m + lane];
                    bit = (__ldg(bm + (col >> 5)) >> (col & 31)) & 1u;
                }
                cnt += __popc(__ballot_sync(kFull, bit != 0u) & rm);
            }
            if (r <= R1 && isS && lo < hi && cnt)
                atomicAdd(&sm.cnt[r - R0], cnt);
            }
        }
    }
    __syncthreads();

    bool fS = false, fE = false, fI = false;
    uint32_t dS = 0;
    if (tid < nrows) {
        const int r = R0 + tid;
        const int64_t rlo = sm.rp[tid], rhi = sm.rp[tid + 1];
        const int x = sm.xs[tid];
        bool do_tail = false;
        uint32_t count = 0;
        float lam = 0.0f;                   // SHED: the row's pressure
        if (x == kS && SHED) {
            if constexpr (SHED) {
                // this chunk's partial: the warps' partials in warp order
                float part = 0.0f;
                for (int w = 0; w < kStepWarps; ++w) {
                    const int d = r - sh.wrow[w];
                    if (d >= 0 && d < kWarp)
                        part = __fadd_rn(part, sh.part[w][d]);
                }
                if (rlo >= e0 && rhi <= e1) {
                    do_tail = true;
                    lam = part;
                } else {
                    // chunk partials land in per-chunk slots; the last chunk
                    // to arrive folds them in chunk order
                    const int64_t cf = rlo / kMergeEPB, cl = (rhi - 1) / kMergeEPB;
                    __stcg(reinterpret_cast<float*>(a.m_part + chunk) + (rlo < e0 ? 0 : 1), part);
                    __threadfence();
                    const uint32_t tk = atomicAdd(a.m_tkt + r, 1u);
                    if (tk == (uint32_t)(cl - cf)) {
                        __threadfence();
                        float tot = __ldcg(reinterpret_cast<const float*>(a.m_part + cf) + 1);
                        for (int64_t c = cf + 1; c <= cl; ++c)
                            tot = __fadd_rn(tot, __ldcg(reinterpret_cast<const float*>(a.m_part + c)));
                        atomicExch(a.m_tkt + r, 0u);
                        do_tail = true;
                        lam = tot;
                    }
                }
            }
        } else if (x == kS) {
            if (rlo >= e0 && rhi <= e1) {
                do_tail = true;
                count = sm.cnt[tid];
            } else {
                const uint32_t nch = (uint32_t)((rhi - 1) / kMergeEPB - rlo / kMergeEPB + 1);
                const uint32_t part = sm.cnt[tid];
                if (part)
                    atomicAdd(reinterpret_cast<unsigned int*>(a.m_cnt + r), part);
                __threadfence();
                const uint32_t tk = atomicAdd(a.m_tkt + r, 1u);
                if (tk == nch - 1u) {
                    __threadfence();
                    count = atomicExch(reinterpret_cast<unsigned int*>(a.m_cnt + r), 0u);
                    atomicExch(a.m_tkt + r, 0u);
                    do_tail = true;
                }
            }
        } else {
            do_tail = rlo >= e0;   // the chunk that holds the row's first edge
        }
        if (do_tail) {
            const int gi = a.m_base + r;
            float age = 0.0f;
            if (x == kE || x == kI)
                age = AgeIO<AgeT>::load(A[gi]);
            TailResult t;
            if constexpr (ADPT) {
                float rate = 0.0f;
                if (x == kS)
                    rate = SHED ? lam : (count ? __fmul_rn(a.M.beta, (float)count) : 0.0f);
                else if (x == kE || x == kI)
                    rate = hazard_of(a.M, x, age);
                lmax = fmaxf(lmax, rate);
                t = tail_p_dt(a, x, age, p_of_rate_dt(rate, dt), gi, step, dt);
            } else if constexpr (SHED) {
                t = tail_p(a, x, age, x == kS ? p_of_rate(a.M, lam) : node_p(a, x, age, 0u), gi, step);
            } else {
                t = tail_at(a, x, age, count, gi, step);
            }
            if (t.x != x)
                a.X[gi] = (uint8_t)t.x;
            if (t.fired || x == kE || x == kI)
                A[gi] = AgeIO<AgeT>::store(t.age);
            if constexpr (SHED) {
                if (t.x == kI)
                    static_cast<AgeT*>(a.rho[(step & 1u) ^ 1u])[gi] =
                        AgeIO<AgeT>::store(rho_of_age(a, AgeIO<AgeT>::load(AgeIO<AgeT>::store(t.age))));
            }
            const int wofs = (gi >> 5) - ((a.m_base + R0) >> 5);
            const uint32_t bit = 1u << (gi & 31);
            if (t.x == kI)
                atomicOr(&sm.wset[wofs], bit);
            else
                atomicOr(&sm.wclr[wofs], bit);
            fS = t.fired && x == kS;
            fE = t.fired && x == kE;
            fI = t.fired && x == kI;
            dS = fS ? (uint32_t)(rhi - rlo) : 0u;
        }
    }
    warp_add_deltas(a.deltas, a.j, fS, fE, fI, dS);
    __syncthreads();
    if (tid < 8) {
        const int w = ((a.m_base + R0) >> 5) + tid;
        if (sm.wset[tid])
            atomicOr(bmn + w, sm.wset[tid]);
        if (sm.wclr[tid])
            atomicAnd(bmn + w, ~sm.wclr[tid]);
    }
}

template <typename AgeT, bool HAS_MERGE, int MODE>
__global__ void __launch_bounds__(kStepThreads, kStepCtasPerSm) fused_step_kernel(const __grid_constant__ StepArgs a)
{
    // Ready for programmatic dependent launch (launch_step's pdl flag): such a
    // grid may start while the previous step drains, so nothing it reads is
    // touched before that grid has completed and flushed (griddepcontrol.wait),
    // and the next step may be scheduled once every CTA of this one has
    // started. Without the launch attribute both instructions do nothing; the
    // step loop launches without it (graph kernel nodes measured faster).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int64_t k = a.ctl->step + a.j;
    const uint32_t par = (uint32_t)(k & 1);
    const uint32_t* __restrict__ bm = a.bm[par];
    uint32_t* __restrict__ bmn = a.bm[par ^ 1u];
    float dt = a.M.dt;
    if constexpr ((MODE & kModeAdaptive) != 0)
        dt = adaptive_dt(a, k);
    LaneDeltas ld;
    bool merge_cta = false;
    if constexpr (HAS_MERGE)
        merge_cta = (int)blockIdx.x < a.n_chunks;
    if (merge_cta) {
        if constexpr (HAS_MERGE)
            merge_chunk<AgeT, MODE>(a, (uint32_t)k, bm, bmn, (int)blockIdx.x, dt, ld.lmax);
    } else {
        const int cta = (int)blockIdx.x - (HAS_MERGE ? a.n_chunks : 0);
        const SliceMap smap = slice_map(a);
        const int s_begin = (cta * kStepWarps + (int)(threadIdx.x >> 5)) * a.spw;
        const int s_end = min(s_begin + a.spw, smap.n_items);
        if (s_begin < s_end) {
            if (smap.list)
                sell_warp<AgeT, MODE, true>(a, (uint32_t)k, bm, bmn, s_begin, s_end, ld, smap, dt);
            else
                sell_warp<AgeT, MODE, false>(a, (uint32_t)k, bm, bmn, s_begin, s_end, ld, smap, dt);
        }
        warp_add_deltas(a.deltas, a.j, ld.fS, ld.fE, ld.fI, ld.dS);
    }
    if constexpr ((MODE & kModeAdaptive) != 0)
        adaptive_lmax(a, k, ld.lmax);
}

// ---------------------------------------------------------------------------
// SELL class with the bitmap in shared memory: one 1024-thread CTA per SM.
// While many nodes are S (the gather-heavy phase), every CTA copies the
// whole current bitmap into shared memory with one bulk TMA copy, overlapped
// with its first state and column loads, and the S lanes' random bit
// gathers hit shared memory instead of L1/L2. Otherwise the gathers read the
// bitmap through the read-only path. Warps take slices round-robin and load
// the next slice's states one iteration ahead.
// ---------------------------------------------------------------------------
// the slice loop of sell_smem_kernel: warps take the slices at positions
// first + j W round-robin (W = resident warps), the states of the next four
// loaded one iteration ahead
template <typename AgeT, int MODE, bool LIST>
__device__ __forceinline__ void smem_slices(const StepArgs& a, uint32_t step, const uint32_t* __restrict__ bm,
                                            const uint32_t* sbm, uint32_t* __restrict__ bmn, bool use_smem,
                                            uint32_t mb, bool& ready, LaneDeltas& ld, const SliceMap& smap,
                                            float dt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = (int)gridDim.x * (kSmemThreads / 32);
    const int first = (int)blockIdx.x * (kSmemThreads / 32) + warp;
    // states of the slices at positions first + (4g + u) W, u = 0..3, packed
    // one byte each
    auto load_group = [&](int base) -> uint32_t {
        uint32_t xs = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int sl = smap.at<LIST>(base + u * W);
            const uint32_t x = (sl < a.n_slices && sl * 32 + lane < a.n_thr) ? (uint32_t)a.X[sl * 32 + lane]
                                                                           : (uint32_t)kR;
            xs |= x << (8 * u);
        }
        return xs;
    };
    uint32_t xs_next = load_group(first);
    for (int base = first; base < smap.n_items; base += 4 * W) {
        const uint32_t xs = xs_next;
        if (base + 4 * W < smap.n_items)
            xs_next = load_group(base + 4 * W);
#pragma unroll 1
        for (int u = 0; u < 4; ++u) {
            const int slice = smap.at<LIST>(base + u * W);
            if (slice >= a.n_slices)
                break;
            const int x = (int)((xs >> (8 * u)) & 0xffu);
            if (__all_sync(kFull, x == kR) && (slice + 1) * 32 <= a.n_thr) {
                if (lane == 0)
                    bmn[slice] = 0u;
                continue;
            }
            if (use_smem)
                sell_slice<AgeT, true, MODE>(a, step, sbm, bmn, slice, x, ld, dt, mb, &ready);
            else
                sell_slice<AgeT, false, MODE>(a, step, bm, bmn, slice, x, ld, dt);
        }
    }
}

template <typename AgeT, int MODE>
__global__ void __launch_bounds__(kSmemThreads, 1) sell_smem_kernel(const __grid_constant__ StepArgs a)
{
    extern __shared__ __align__(128) uint32_t sbm[];
    __shared__ __align__(8) unsigned long long mbar;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int tid = threadIdx.x;
    const int64_t k = a.ctl->step + a.j;
    const uint32_t par = (uint32_t)(k & 1);
    const uint32_t* __restrict__ bm = a.bm[par];
    uint32_t* __restrict__ bmn = a.bm[par ^ 1u];
    const bool use_smem = a.ctl->counts[0] >= a.smem_min_s;
    const uint32_t mb = smem_addr(&mbar);
    if (use_smem && tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(a.bm_bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(sbm)),
                     "l"(bm), "r"(a.bm_bytes), "r"(mb)
                     : "memory");
    }
    __syncthreads();
    LaneDeltas ld;
    bool ready = !use_smem;
    float dt = a.M.dt;
    if constexpr ((MODE & kModeAdaptive) != 0)
        dt = adaptive_dt(a, k);
    const SliceMap smap = slice_map(a);
    if (smap.list)
        smem_slices<AgeT, MODE, true>(a, (uint32_t)k, bm, sbm, bmn, use_smem, mb, ready, ld, smap, dt);
    else
        smem_slices<AgeT, MODE, false>(a, (uint32_t)k, bm, sbm, bmn, use_smem, mb, ready, ld, smap, dt);
    if constexpr ((MODE & kModeAdaptive) != 0)
        adaptive_lmax(a, k, ld.lmax);
    // the copy into this CTA's shared memory must have landed before it exits
    if (!ready && !mbar_wait(mb, 0u, a.wait_limit ? a.wait_limit : kWaitLimit))
        record_error(a.ctl, kErrTmaTimeout);
    warp_add_deltas(a.deltas, a.j, ld.fS, ld.fE, ld.fI, ld.dS);
}

// Memoised Bernoulli probabilities of one sim: the fixed-step age sequence
// a_0 = 0, a_{n+1} = store(a_n + dt) is generated by one thread (it is
// sequential), which also assigns each distinct age its slot at the index the
// step computes from the age (the sequence is monotone, so the ages sharing
// an index are consecutive; with FP16/BF16 storage two can share one, and a
// third would be evaluated directly by the step); then every entry is
// evaluated in parallel with the step's own hazard code. Unfilled slots hold
// NaN ages.
__global__ void build_ptables_kernel(ModelF M, int age_dtype, float4* __restrict__ tab, float* __restrict__ ps,
                                     float4* __restrict__ rtab, LawF shed, int shed_mode)
{
    __shared__ float ages[kPTableN];
    if (threadIdx.x == 0) {
        float v = 0.0f;
        for (int n = 0; n < kPTableN; ++n) {
            ages[n] = v;
            v = age_step_stored(v, M.dt, age_dtype);
        }
    }
    __syncthreads();
    for (int n = threadIdx.x; n < kPTableN; n += blockDim.x) {
        const float v = ages[n];
        const int idx = __float2int_rn(__fmul_rn(v, M.inv_dt));
        // slot = distinct earlier ages with the same index (a repeated age,
        // one that freezes in storage, already has its slot)
        int sl = -1;
        if (n == 0 || ages[n - 1] != v) {
            sl = 0;
            for (int m = n - 1; m >= 0 && __float2int_rn(__fmul_rn(ages[m], M.inv_dt)) == idx && sl < 2; --m)
                if (ages[m] != ages[m + 1])
                    ++sl;
            if (sl >= 2)
                sl = -1;
        }
        if (sl >= 0 && idx >= 0 && idx < kPTableN) {
            float* lat = reinterpret_cast<float*>(tab + idx) + 2 * sl;
            float* inf = reinterpret_cast<float*>(tab + kPTableN + idx) + 2 * sl;
            lat[0] = v;
            lat[1] = p_of_rate(M, hazard(M.lat, v));
            inf[0] = v;
            inf[1] = p_of_rate(M, hazard(M.inf, v));
            if (rtab) {
                float* rr = reinterpret_cast<float*>(rtab + idx) + 2 * sl;
                rr[0] = v;
                rr[1] = shed_value(shed, shed_mode, M.beta, v);
            }
        }
    }
    for (int c = threadIdx.x; c < kPSTableN; c += blockDim.x)
        ps[c] = p_of_rate(M, __fmul_rn(M.beta, (float)c));
}

// ---------------------------------------------------------------------------
// Run bookkeeping: begin (row 0 of the counts output) and the epilogue that
// integrates K steps of deltas into counts (one launch per K steps).
// ---------------------------------------------------------------------------
__global__ void run_begin_kernel(DevCtl* ctl, uint32_t* out)
{
    if (threadIdx.x == 0) {
        ctl->out = out;
        ctl->row = 0;
        if (out) {
            for (int t = 0; t < 4; ++t)
                out[t] = ctl->counts[t];
            ctl->row = 1;
        }
    }
}

static_assert(kDeltaSlots == 32, "the epilogue sums one delta slot per lane");

__global__ void run_epilogue_kernel(DevCtl* ctl, unsigned long long* deltas, int K, int model, const float* dtrec,
                                    float dt)
{
    __shared__ unsigned long long d[kMaxGraphSteps][kDeltaFields];
    // warp w sums the slots of steps w, w + warps, ... (lane = slot) and
    // clears them for the next launch sequence
    const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    for (int j = (int)(threadIdx.x >> 5); j < K; j += nw) {
        ulonglong2* row = reinterpret_cast<ulonglong2*>(deltas + (int64_t)j * kDeltaRow + lane * kDeltaFields);
        const ulonglong2 v0 = row[0], v1 = row[1];
        row[0] = make_ulonglong2(0ull, 0ull);
        row[1] = make_ulonglong2(0ull, 0ull);
        unsigned long long f[kDeltaFields] = {v0.x, v0.y, v1.x, v1.y};
#pragma unroll
        for (int q = 0; q < kDeltaFields; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                f[q] += __shfl_xor_sync(kFull, f[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < kDeltaFields; ++q)
                d[j][q] = f[q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t c0 = ctl->counts[0], c1 = ctl->counts[1], c2 = ctl->counts[2], c3 = ctl->counts[3];
        unsigned long long ds = ctl->ds_cur, dst = ctl->ds_total, st = ctl->s_total, trans = ctl->transitions;
        uint32_t* out = ctl->out;
        const int64_t row = ctl->row;
        for (int j = 0; j < K; ++j) {
            st += c0;
            dst += ds;
            const uint32_t l = (uint32_t)d[j][0], ei = (uint32_t)d[j][1], ir = (uint32_t)d[j][2];
            trans += (unsigned long long)l + ei + ir;
            c0 -= l;
            if (model == kSEIR) {
                c1 += l - ei;
                c2 += ei - ir;
                c3 += ir;
            } else if (model == kSIS) {           // recoveries return to S
                c0 += ir;
                c2 += l - ir;
            } else {
                c2 += l - ir;
                c3 += ir;
            }
            ds -= d[j][3];
            if (out) {
                uint32_t* o = out + (row + j) * 4;
                o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
            }
        }
        ctl->counts[0] = c0; ctl->counts[1] = c1; ctl->counts[2] = c2; ctl->counts[3] = c3;
        ctl->ds_cur = ds;
        ctl->transitions = trans;
        ctl->ds_total = dst;
        ctl->s_total = st;
        double t = ctl->time;
        for (int j = 0; j < K; ++j)
            t += (double)(dtrec ? dtrec[j] : dt);
        ctl->time = t;
        ctl->act_sum += ctl->n_act;
        ctl->n_act = 0ull;                 // the next launch sequence's refresh counts from 0
        ctl->step += K;
        if (out)
            ctl->row = row + K;
    }
}

// Rebuild the infectious bitmap of the current step parity, the counts and
// the S-degree sum from the state (after init or set_state).
__global__ void refresh_kernel(const uint8_t* __restrict__ X, int n, const int32_t* __restrict__ deg,
                               uint32_t* bm0, uint32_t* bm1, DevCtl* ctl)
{
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int i = w * 32 + lane;
    const int x = (i < n) ? (int)X[i] : -1;
    const uint32_t word = __ballot_sync(kFull, x == kI);
    const unsigned long long dS = (x == kS) ? (unsigned long long)deg[i] : 0ull;
    uint32_t cs[4];
    for (int c = 0; c < 4; ++c)
        cs[c] = __popc(__ballot_sync(kFull, x == c));
    unsigned long long dsum = dS;
    for (int o = 16; o > 0; o >>= 1)
        dsum += __shfl_xor_sync(kFull, dsum, o);
    if (lane == 0 && w * 32 < n) {
        const uint32_t par = (uint32_t)(ctl->step & 1);
        (par ? bm1 : bm0)[w] = word;
        for (int c = 0; c < 4; ++c)
            if (cs[c])
                atomicAdd(&ctl->counts[c], cs[c]);
        if (dsum)
            atomicAdd(&ctl->ds_cur, dsum);
    }
}

__global__ void set_index_kernel(uint8_t* X, const int32_t* idx, int64_t n_idx, const int32_t* inv, int state)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n_idx) {
        const int o = idx[q];
        X[inv ? inv[o] : o] = (uint8_t)state;
    }
}

// out[perm[i]] = in[i] (internal -> original order), elements of `bytes`
template <typename T>
__global__ void to_original_kernel(const T* __restrict__ in, T* __restrict__ out, const int32_t* perm, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[perm[i]] = in[i];
}

template <typename T>
__global__ void from_original_kernel(const T* __restrict__ in, T* __restrict__ out, const int32_t* inv, int n)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < n)
        out[inv[o]] = in[o];
}

// Active-node compaction refresh (Section 5.6) for the gather form, at the
// start of a launch sequence: lists the SELL slices that still hold a non-R
// node (the last slice, whose bitmap word merge-class nodes may share, is
// always listed) and clears both bitmap words of the others, which the steps
// will no longer write (their nodes are R: no infectious bit can appear).
// While fewer than half the nodes are R it writes "all slices" instead.
// ctl->n_act is 0 on entry.
__global__ void sell_compact_kernel(const __grid_constant__ StepArgs a)
{
    if ((int64_t)a.ctl->counts[3] * 2 < (int64_t)a.n) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            a.ctl->n_act = (unsigned long long)a.n_slices;
        return;
    }
    const int lane = threadIdx.x & 31;
    const int stride = (int)(gridDim.x * blockDim.x);
    for (int t0 = (int)(blockIdx.x * blockDim.x) + (int)(threadIdx.x & ~31u); t0 < a.n_slices; t0 += stride) {
        const int t = t0 + lane;
        bool live = false;
        if (t < a.n_slices) {
            if ((t + 1) * 32 > a.n_thr) {
                live = true;
            } else {
                const uint4 x0 = *reinterpret_cast<const uint4*>(a.X + (int64_t)t * 32);
                const uint4 x1 = *reinterpret_cast<const uint4*>(a.X + (int64_t)t * 32 + 16);
                live = (x0.x & x0.y & x0.z & x0.w & x1.x & x1.y & x1.z & x1.w) != 0x03030303u;
                if (!live) {
                    a.bm[0][t] = 0u;
                    a.bm[1][t] = 0u;
                }
            }
        }
        const uint32_t b = __ballot_sync(kFull, live);
        if (b) {
            unsigned long long base = 0ull;
            if (lane == 0)
                base = atomicAdd(&a.ctl->n_act, (unsigned long long)__popc(b));
            base = __shfl_sync(kFull, base, 0);
            if (live)
                a.act[base + __popc(b & ((1u << lane) - 1u))] = t;
        }
    }
}

// infectivity of the I nodes at the current step (after init or set_state)
template <typename AgeT>
__global__ void rho_init_kernel(const __grid_constant__ StepArgs a, uint32_t par)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n && a.X[i] == kI) {
        const float age = AgeIO<AgeT>::load(static_cast<const AgeT*>(a.A)[i]);
        static_cast<AgeT*>(a.rho[par])[i] = AgeIO<AgeT>::store(shed_rho(a, age));
    }
}

__global__ void eval_density_kernel(LawF L, const float* tau, float* f, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        f[i] = density(L, tau[i]);
}

__global__ void eval_hazard_kernel(LawF L, const float* tau, float* h, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        h[i] = hazard(L, tau[i]);
}

__global__ void eval_uniform_kernel(uint32_t key0, uint32_t key1, uint32_t rep, uint32_t step,
                                    const int32_t* nodes, float* u, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        u[i] = uniform24(key0, key1, rep, step, (uint32_t)nodes[i]);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename AgeT>
static cudaError_t launch_step_t(const StepArgs& a, cudaStream_t s, bool pdl)
{
    const int grid = a.n_chunks + a.n_sell_ctas;
    if (grid == 0)
        return cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kStepThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e;
    const int mode = (a.shed_mode != kShedNone ? kModeShed : 0) | (a.dtrec ? kModeAdaptive : 0);
    if (a.n_chunks > 0) {
        switch (mode) {
        case 1: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, true, 1>, a); break;
        case 2: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, true, 2>, a); break;
        case 3: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, true, 3>, a); break;
        default: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, true, 0>, a); break;
        }
    } else {
        switch (mode) {
        case 1: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, false, 1>, a); break;
        case 2: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, false, 2>, a); break;
        case 3: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, false, 3>, a); break;
        default: e = cudaLaunchKernelEx(&cfg, fused_step_kernel<AgeT, false, 0>, a); break;
        }
    }
    g_launch_count += 1;
    return e;
}

cudaError_t launch_step(const StepArgs& a, int age_dtype, cudaStream_t s, bool pdl)
{
    switch (age_dtype) {
    case kAgeF16: return launch_step_t<__half>(a, s, pdl);
    case kAgeBF16: return launch_step_t<__nv_bfloat16>(a, s, pdl);
    default: return launch_step_t<float>(a, s, pdl);
    }
}

template <typename AgeT>
static cudaError_t launch_step_smem_t(const StepArgs& a, cudaStream_t s, int num_sms)
{
    static thread_local int configured = 0;   // dynamic shared memory limits set once per thread
    if (!configured) {
        cudaError_t e = cudaSuccess;
        for (auto f : {sell_smem_kernel<AgeT, 0>, sell_smem_kernel<AgeT, 1>, sell_smem_kernel<AgeT, 2>,
                       sell_smem_kernel<AgeT, 3>})
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBitmapMaxBytes);
        if (e != cudaSuccess)
            return e;
        configured = 1;
    }
    const int grid = std::max(1, std::min(num_sms, (a.n_slices + 31) / 32));
    switch ((a.shed_mode != kShedNone ? kModeShed : 0) | (a.dtrec ? kModeAdaptive : 0)) {
    case 1: sell_smem_kernel<AgeT, 1><<<grid, kSmemThreads, a.bm_bytes, s>>>(a); break;
    case 2: sell_smem_kernel<AgeT, 2><<<grid, kSmemThreads, a.bm_bytes, s>>>(a); break;
    case 3: sell_smem_kernel<AgeT, 3><<<grid, kSmemThreads, a.bm_bytes, s>>>(a); break;
    default: sell_smem_kernel<AgeT, 0><<<grid, kSmemThreads, a.bm_bytes, s>>>(a); break;
    }
    g_launch_count += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n_chunks == 0)
        return e;
    // merge class of the same step (independent of the SELL class) in a second grid
    StepArgs m = a;
    m.n_sell_ctas = 0;
    return launch_step_t<AgeT>(m, s, false);
}

cudaError_t launch_step_smem(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms)
{
    switch (age_dtype) {
    case kAgeF16: return launch_step_smem_t<__half>(a, s, num_sms);
    case kAgeBF16: return launch_step_smem_t<__nv_bfloat16>(a, s, num_sms);
    default: return launch_step_smem_t<float>(a, s, num_sms);
    }
}

cudaError_t launch_build_ptables(const ModelF& M, int age_dtype, float4* tab, float* ps, cudaStream_t s,
                                 float4* rtab, const LawF& shed, int shed_mode)
{
    build_ptables_kernel<<<1, 256, 0, s>>>(M, age_dtype, tab, ps, rtab, shed, shed_mode);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_run_begin(DevCtl* ctl, uint32_t* out, cudaStream_t s)
{
    run_begin_kernel<<<1, 32, 0, s>>>(ctl, out);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_run_epilogue(DevCtl* ctl, unsigned long long* deltas, int K, int model, const float* dtrec,
                                float dt, cudaStream_t s)
{
    run_epilogue_kernel<<<1, 1024, 0, s>>>(ctl, deltas, K, model, dtrec, dt);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_refresh(const uint8_t* X, int n, const int32_t* deg, uint32_t* bm0, uint32_t* bm1, DevCtl* ctl,
                           cudaStream_t s)
{
    const int words = (n + 31) / 32;
    const int threads = 256;
    const int blocks = (int)(((int64_t)words * 32 + threads - 1) / threads);
    refresh_kernel<<<blocks, threads, 0, s>>>(X, n, deg, bm0, bm1, ctl);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_set_index(uint8_t* X, const int32_t* idx, int64_t n_idx, const int32_t* inv, int state,
                             cudaStream_t s)
{
    if (n_idx == 0)
        return cudaSuccess;
    set_index_kernel<<<(unsigned)((n_idx + 255) / 256), 256, 0, s>>>(X, idx, n_idx, inv, state);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_to_original(const void* in, void* out, int elem_bytes, const int32_t* perm, int n, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (elem_bytes == 1)
        to_original_kernel<uint8_t><<<blocks, 256, 0, s>>>((const uint8_t*)in, (uint8_t*)out, perm, n);
    else if (elem_bytes == 2)
        to_original_kernel<uint16_t><<<blocks, 256, 0, s>>>((const uint16_t*)in, (uint16_t*)out, perm, n);
    else
        to_original_kernel<uint32_t><<<blocks, 256, 0, s>>>((const uint32_t*)in, (uint32_t*)out, perm, n);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_from_original(const void* in, void* out, int elem_bytes, const int32_t* inv, int n,
                                 cudaStream_t s)
{
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (elem_bytes == 1)
        from_original_kernel<uint8_t><<<blocks, 256, 0, s>>>((const uint8_t*)in, (uint8_t*)out, inv, n);
    else if (elem_bytes == 2)
        from_original_kernel<uint16_t><<<blocks, 256, 0, s>>>((const uint16_t*)in, (uint16_t*)out, inv, n);
    else
        from_original_kernel<uint32_t><<<blocks, 256, 0, s>>>((const uint32_t*)in, (uint32_t*)out, inv, n);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_sell_compact(const StepArgs& a, cudaStream_t s, int num_sms)
{
    const int need = (a.n_slices + 255) / 256;
    const int grid = std::max(1, std::min(need, num_sms * 8));
    sell_compact_kernel<<<grid, 256, 0, s>>>(a);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_rho_init(const StepArgs& a, int age_dtype, uint32_t par, cudaStream_t s)
{
    if (a.n == 0)
        return cudaSuccess;
    const int blocks = (a.n + 255) / 256;
    switch (age_dtype) {
    case kAgeF16: rho_init_kernel<__half><<<blocks, 256, 0, s>>>(a, par); break;
    case kAgeBF16: rho_init_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(a, par); break;
    default: rho_init_kernel<float><<<blocks, 256, 0, s>>>(a, par); break;
    }
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_eval_density(const LawF& L, const float* tau, float* f, int64_t n, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    eval_density_kernel<<<(unsigned)blocks, 256, 0, s>>>(L, tau, f, n);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_eval_hazard(const LawF& L, const float* tau, float* h, int64_t n, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    eval_hazard_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, tau, h, n);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_eval_uniforms(uint32_t key0, uint32_t key1, uint32_t rep, uint32_t step, const int32_t* nodes,
                                 float* u, int64_t n, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    eval_uniform_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(key0, key1, rep, step, nodes, u, n);
    g_launch_count += 1;
    return cudaGetLastError();
}

}  // namespace fs
