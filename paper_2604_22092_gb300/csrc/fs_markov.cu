// fs_markov.cu -- the Markovian engine of FlashSpread (arXiv 2604.22092),
// Section 4, Algorithm 1: constant rates (S: beta x infectious in-neighbours,
// E: sigma, I: gamma), one tau-leaping step of size
//   tau = min(theta N / Lambda, p_max / max_i lambda_i, tau_max)
// from the rates of the current state, then Bernoulli(1 - exp(-lambda_i tau))
// transitions (SIS: I -> S; SIR / SEIR: I -> R), then the infection counts of
// the next state: by +-1 atomics along the transposed CSR from the nodes that
// entered or left I (Inertial Mode) or by a dense recount over the rows
// (Control Mode), whichever touches less memory. The counts are integers, so
// both modes give the same counts and no periodic recomputation is needed.
//
// One step = three launches: rates (integer reductions of the current state
// into the control block), step (tau, draws, transitions, event list),
// influence (counts of the next state).
#include <cuda_runtime.h>

#include <algorithm>

#include "fs_device.cuh"
#include "fs_launch.h"

namespace fs {

namespace {

constexpr int kMkThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ void mk_record_error(DevCtl* ctl, int code)
{
    atomicCAS(&ctl->error, 0, code);
}

// Rates of the current state, reduced to integers so that Lambda and the
// largest rate (and hence tau) are exact and schedule-independent:
// Lambda = beta * (S-I edges) + sigma * |E| + gamma * |I|,
// max lambda = max(beta * max_S c, sigma [|E| > 0], gamma [|I| > 0]).
__global__ void __launch_bounds__(kMkThreads) mk_rates_kernel(const __grid_constant__ StepArgs a)
{
    __shared__ unsigned long long s_si, s_ne, s_ni;
    __shared__ unsigned int s_cmax;
    const int64_t k = a.ctl->step + a.j;
    MarkovSums* out = &a.ctl->mk[k & 1];
    if (threadIdx.x == 0) {
        s_si = s_ne = s_ni = 0ull;
        s_cmax = 0u;
        if (blockIdx.x == 0)
            a.ctl->mk_nev = 0u;            // the step appends this step's events from 0
    }
    __syncthreads();
    unsigned long long si = 0ull, ne = 0ull, ni = 0ull;
    unsigned int cmax = 0u;
    // four consecutive nodes per thread: one 4-byte state load, and one
    // 16-byte count load when one of them is S (the buffers are padded to 16
    // nodes; padding reads as S with count 0 and is skipped)
    const int64_t n_grp = ((int64_t)a.n + 3) / 4;
    for (int64_t q = (int64_t)blockIdx.x * kMkThreads + threadIdx.x; q < n_grp;
         q += (int64_t)gridDim.x * kMkThreads) {
        const int64_t i0 = q * 4;
        const uint32_t xw = *reinterpret_cast<const uint32_t*>(a.X + i0);
        uint4 cw = make_uint4(0u, 0u, 0u, 0u);
        if (__vcmpeq4(xw, 0u))
            cw = *reinterpret_cast<const uint4*>(a.mk_cnt + i0);
        const unsigned int cs[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i0 + u < a.n) {
                const int x = (int)((xw >> (8 * u)) & 0xffu);
                if (x == kS) {
                    si += cs[u];
                    cmax = max(cmax, cs[u]);
                } else if (x == kE) {
                    ne += 1ull;
                } else if (x == kI) {
                    ni += 1ull;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        si += __shfl_down_sync(kFull, si, o);
    ne = __reduce_add_sync(kFull, (unsigned)ne);     // node counts fit 32 bits
    ni = __reduce_add_sync(kFull, (unsigned)ni);
    cmax = __reduce_max_sync(kFull, cmax);
    if ((threadIdx.x & 31) == 0) {
        if (si) atomicAdd(&s_si, si);
        if (ne) atomicAdd(&s_ne, ne);
        if (ni) atomicAdd(&s_ni, ni);
        if (cmax) atomicMax(&s_cmax, cmax);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_si) atomicAdd(&out->si, s_si);
        if (s_ne) atomicAdd(&out->ne, s_ne);
        if (s_ni) atomicAdd(&out->ni, s_ni);
        if (s_cmax) atomicMax(&out->cmax, s_cmax);
    }
}

// Algorithm 1's step size, in double in the oracle's order, as the float the
// ages advance by. Every thread computes the same value.
__device__ __forceinline__ float mk_tau(const StepArgs& a, const MarkovSums& m)
{
    const double lam = __dadd_rn(__dadd_rn(__dmul_rn(a.mk_beta, (double)m.si), __dmul_rn(a.mk_sigma, (double)m.ne)),
                                 __dmul_rn(a.mk_gamma, (double)m.ni));
    double lmax = __dmul_rn(a.mk_beta, (double)m.cmax);
    if (m.ne > 0ull && a.mk_sigma > lmax)
        lmax = a.mk_sigma;
    if (m.ni > 0ull && a.mk_gamma > lmax)
        lmax = a.mk_gamma;
    double tau = a.mk_tau_max;
    if (lam > 0.0) {
        const double t1 = __ddiv_rn(__dmul_rn(a.mk_theta, (double)a.n), lam);
        if (t1 < tau)
            tau = t1;
    }
    if (lmax > 0.0) {
        const double t2 = __ddiv_rn(a.mk_p_max, lmax);
        if (t2 < tau)
            tau = t2;
    }
    return (float)tau;
}

// Draws and transitions of one step; nodes entering or leaving I are
// appended to the event list (node | bit 31 when it left I).
template <typename AgeT>
__global__ void __launch_bounds__(kMkThreads) mk_step_kernel(const __grid_constant__ StepArgs a)
{
    __shared__ float s_tau;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t k = a.ctl->step + a.j;
    // tau once per block: double arithmetic is slow on this part, and every
    // thread would compute the same value
    if (tid == 0) {
        s_tau = mk_tau(a, a.ctl->mk[k & 1]);
        if (blockIdx.x == 0) {
            a.dtrec[a.j] = s_tau;
            a.ctl->mk[(k + 1) & 1] = MarkovSums{};   // for the next step's reduction
        }
    }
    __syncthreads();
    const float tau = s_tau;
    AgeT* __restrict__ A = static_cast<AgeT*>(a.A);
    const int model = a.M.model;
    uint32_t fS = 0u, fE = 0u, fI = 0u;
    unsigned long long dS = 0ull;          // net change of the S-degree sum, modulo 2^64
    const int64_t stride = (int64_t)gridDim.x * kMkThreads;
    // four consecutive nodes per thread (independent chains of loads and
    // draws); the buffers are padded to 16 nodes, padding is never written
    const int64_t n_grp = ((int64_t)a.n + 3) / 4;
    for (int64_t q0 = (int64_t)blockIdx.x * kMkThreads + (tid & ~31); q0 < n_grp; q0 += stride) {
        const int64_t q = q0 + lane;
        uint32_t evm = 0u, leftm = 0u;
        if (q < n_grp) {
            const int64_t i0 = q * 4;
            const uint32_t xw = *reinterpret_cast<const uint32_t*>(a.X + i0);
            uint4 cw = make_uint4(0u, 0u, 0u, 0u);
            if (__vcmpeq4(xw, 0u))
                cw = *reinterpret_cast<const uint4*>(a.mk_cnt + i0);
            const unsigned int cs[4] = {cw.x, cw.y, cw.z, cw.w};
            uint32_t yw = xw;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = i0 + u;
                if (i >= a.n)
                    continue;
                const int x = (int)((xw >> (8 * u)) & 0xffu);
                float lam = 0.0f;
                if (x == kS)
                    lam = cs[u] ? __fmul_rn(a.M.beta, (float)cs[u]) : 0.0f;
                else if (x == kE)
                    lam = a.M.lat.p0;
                else if (x == kI)
                    lam = a.M.inf.p0;
                bool fired = false;
                if (lam > 0.0f) {
                    const float p = -expm1f(-__fmul_rn(lam, tau));
                    const uint32_t node = a.perm ? (uint32_t)__ldg(a.perm + i) : (uint32_t)i;
                    fired = uniform24(a.M.key0, a.M.key1, a.M.rep, (uint32_t)k, node) < p;
                }
                int y = x;
                if (fired)
                    y = x == kS ? (model == kSEIR ? kE : kI) : x == kE ? kI : (model == kSIS ? kS : kR);
                if (y != x)
                    yw = (yw & ~(0xffu << (8 * u))) | ((uint32_t)y << (8 * u));
                if (fired || x == kE || x == kI) {
                    const float age = fired ? 0.0f : __fadd_rn(AgeIO<AgeT>::load(A[i]), tau);
                    A[i] = AgeIO<AgeT>::store(age);
                }
                if (fired) {
                    fS += x == kS;
                    fE += x == kE;
                    fI += x == kI;
                    const unsigned long long d = (unsigned long long)__ldg(a.deg + i);
                    if (x == kS)
                        dS += d;
                    else if (y == kS)
                        dS -= d;
                }
                if ((x == kI) != (y == kI)) {
                    evm |= 1u << u;
                    if (x == kI)
                        leftm |= 1u << u;
                }
            }
            if (yw != xw)
                *reinterpret_cast<uint32_t*>(a.X + i0) = yw;
        }
        // nodes that entered or left I go to the event list
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ev = (evm >> u) & 1u;
            const uint32_t b = __ballot_sync(kFull, ev);
            if (b) {
                unsigned int base = 0u;
                if (lane == 0)
                    base = atomicAdd(&a.ctl->mk_nev, (unsigned int)__popc(b));
                base = __shfl_sync(kFull, base, 0);
                if (ev)
                    a.mk_ev[base + __popc(b & ((1u << lane) - 1u))] =
                        (uint32_t)(q * 4 + u) | (((leftm >> u) & 1u) ? 0x80000000u : 0u);
            }
        }
    }
    warp_add_deltas(a.deltas, a.j, fS, fE, fI, dS);
}

// Control Mode: every node's count recomputed from its row. Warps take
// work items: SELL slices (one lane per node, the slice's columns) and then
// merge-class rows (the warp strides over the row).
__device__ __forceinline__ void mk_recount_item(const StepArgs& a, int64_t w, int lane)
{
    if (w < a.n_slices) {
        const int s = (int)w;
        const int64_t off = __ldg(a.sell_off + s);
        const int width = (int)((__ldg(a.sell_off + s + 1) - off) >> 5);
        const int i = s * 32 + lane;
        unsigned int c = 0u;
        for (int t = 0; t < width; ++t) {
            const int j = __ldg(a.sell_col + off + 32 * t + lane);
            if (j < a.n && a.X[j] == kI)
                c += 1u;
        }
        if (i < a.n_thr)
            a.mk_cnt[i] = c;
    } else if (w < a.n_slices + a.n_m) {
        const int r = (int)(w - a.n_slices);
        const int64_t lo = __ldg(a.m_ptr + r), hi = __ldg(a.m_ptr + r + 1);
        unsigned int c = 0u;
        for (int64_t e = lo + lane; e < hi; e += 32) {
            const int j = __ldg(a.m_col + e);
            if (j < a.n && a.X[j] == kI)
                c += 1u;
        }
        c = __reduce_add_sync(kFull, c);
        if (lane == 0)
            a.mk_cnt[a.n_thr + r] = c;
    }
}

// Counts of the next state: Inertial Mode (+-1 along the transposed rows of
// the event nodes, a warp per event) unless the events' out-edges outnumber
// a quarter of all edges, then Control Mode. mode_force: 1 always inertial,
// 2 always control, 0 by that rule.
__global__ void __launch_bounds__(kMkThreads) mk_influence_kernel(const __grid_constant__ StepArgs a, int recount_only)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kMkThreads + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * kMkThreads) >> 5;
    bool control = recount_only != 0;
    int64_t n_ev = 0;
    if (!control) {
        n_ev = (int64_t)a.ctl->mk_nev;
        if (n_ev > a.n) {                       // cannot happen: one event per node per step
            mk_record_error(a.ctl, kErrBadState);
            return;
        }
        control = a.mk_mode == 2 ||
                  (a.mk_mode == 0 && (double)n_ev * a.mk_avg_deg * 4.0 > (double)a.e_total);
    }
    if (control) {
        for (int64_t w = warp; w < (int64_t)a.n_slices + a.n_m; w += n_warps)
            mk_recount_item(a, w, lane);
        return;
    }
    for (int64_t e = warp; e < n_ev; e += n_warps) {
        const uint32_t v = a.mk_ev[e];
        const uint32_t j = v & 0x7fffffffu;
        const int delta = (v >> 31) ? -1 : 1;
        const int64_t lo = __ldg(a.out_ptr + j), hi = __ldg(a.out_ptr + j + 1);
        for (int64_t q = lo + lane; q < hi; q += 32)
            atomicAdd(a.mk_cnt + __ldg(a.out_col + q), (unsigned int)delta);
    }
}

template <typename AgeT>
cudaError_t launch_mk_step_t(const StepArgs& a, cudaStream_t s, int num_sms)
{
    const int64_t need = (((int64_t)a.n + 3) / 4 + kMkThreads - 1) / kMkThreads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * 8));
    mk_rates_kernel<<<grid, kMkThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    mk_step_kernel<AgeT><<<grid, kMkThreads, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int64_t items = (int64_t)a.n_slices + a.n_m;
    const int grid_i = (int)std::max<int64_t>(
        1, std::min<int64_t>((items * 32 + kMkThreads - 1) / kMkThreads, (int64_t)num_sms * 8));
    mk_influence_kernel<<<grid_i, kMkThreads, 0, s>>>(a, 0);
    g_launch_count += 3;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_markov_step(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms)
{
    switch (age_dtype) {
    case kAgeF16: return launch_mk_step_t<__half>(a, s, num_sms);
    case kAgeBF16: return launch_mk_step_t<__nv_bfloat16>(a, s, num_sms);
    default: return launch_mk_step_t<float>(a, s, num_sms);
    }
}

cudaError_t launch_markov_recount(const StepArgs& a, cudaStream_t s, int num_sms)
{
    const int64_t items = (int64_t)a.n_slices + a.n_m;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((items * 32 + kMkThreads - 1) / kMkThreads, (int64_t)num_sms * 8));
    mk_influence_kernel<<<grid, kMkThreads, 0, s>>>(a, 1);
    g_launch_count += 1;
    return cudaGetLastError();
}

}  // namespace fs
