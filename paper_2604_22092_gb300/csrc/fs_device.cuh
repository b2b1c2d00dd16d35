// fs_device.cuh -- device building blocks of the fused renewal step:
// Philox4x32-10 uniforms, FP32 hazards, and the per-node tail (hazard ->
// Bernoulli -> transition -> renewal age) of FlashSpread (arXiv 2604.22092),
// Algorithm 3 at a fixed step.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fs_internal.h"

namespace fs {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor bijection on a 128-bit counter under a 64-bit key bumped by
// the two Weyl constants between rounds. Replaces the paper's
// tl.rand(seed + step_id, node_id) (Appendix A) with a draw keyed by
// (seed, replicate, step, node) so that every traversal class, packing and
// batching draws the same number for the same node-step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        // one 32 x 32 -> 64-bit product gives both halves of each multiply
        const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// u = (w >> 8) * 2^-24, exactly representable in FP32.
__device__ __forceinline__ float uniform24(uint32_t key0, uint32_t key1, uint32_t rep,
                                           uint32_t step, uint32_t node)
{
    const uint4 w = philox4x32_10(make_uint4(node, step, rep >> 2, 0u), key0, key1);
    const uint32_t sel = rep & 3u;
    const uint32_t word = sel == 0 ? w.x : sel == 1 ? w.y : sel == 2 ? w.z : w.w;
    return (float)(word >> 8) * 5.9604644775390625e-08f;
}

// ---------------------------------------------------------------------------
// Hazards in FP32 (Section 5.1; Proposition 1 for the log-normal).
//
// The log-normal hazard h = sqrt(2/pi) / (tau sigma erfcx(z)) is
// exponentially sensitive to z when z << 0 (young ages): its relative error
// is about 2|z| times the absolute error of z. So z = (ln tau - mu) /
// (sigma sqrt 2) is formed as an unevaluated float pair (error-free sums and
// fma products; ln tau = e ln2 + log1p(m - 1) with ln2 split in two), and for
// z < -2 the hazard is evaluated as sqrt(2/pi)/sigma * e^{-z^2} / (tau
// erfc(z)) with z^2 split exactly, erfc(z) = 2 - erfc(-z). For z >= -2 the
// CUDA erfcxf of the rounded z is accurate enough. Every operation is FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// z = (ln tau - mu) / (sigma sqrt 2) as an unevaluated pair zh + zl (tau > 0)
__device__ __forceinline__ void lognormal_z(const LawF& L, float tau, float& zh, float& zl)
{
    constexpr float kLn2Hi = 0.693145751953125f;          // ln 2 to 16 bits (e * kLn2Hi is exact)
    constexpr float kLn2Lo = 1.4286067653302226e-06f;     // ln 2 - kLn2Hi
    int e;
    float m = frexpf(tau, &e);                            // tau = m 2^e, m in [0.5, 1)
    if (m < 0.70710678f) {
        m = m * 2.0f;
        e -= 1;
    }
    const float lm = log1pf(__fsub_rn(m, 1.0f));          // m - 1 is exact
    float a_hi, a_lo;
    two_sum(__fmul_rn((float)e, kLn2Hi), lm, a_hi, a_lo);
    a_lo = __fadd_rn(a_lo, __fmul_rn((float)e, kLn2Lo));
    float d_hi, d_lo;
    two_sum(a_hi, -L.p0, d_hi, d_lo);                     // ln tau - mu
    d_lo = __fadd_rn(d_lo, __fsub_rn(a_lo, L.p3));
    const float z_hi = __fmul_rn(d_hi, L.p1);
    const float z_lo = __fadd_rn(__fmaf_rn(d_hi, L.p1, -z_hi),
                                 __fadd_rn(__fmul_rn(d_hi, L.p4), __fmul_rn(d_lo, L.p1)));
    zh = __fadd_rn(z_hi, z_lo);
    zl = __fsub_rn(z_lo, __fsub_rn(zh, z_hi));
}

// e^{-z^2} for z = zh + zl, with z^2 split exactly
__device__ __forceinline__ float exp_neg_z2(float zh, float zl)
{
    const float s_hi = __fmul_rn(zh, zh);
    const float s_lo = __fadd_rn(__fmaf_rn(zh, zh, -s_hi), __fmul_rn(__fmul_rn(2.0f, zh), zl));
    return __fmul_rn(expf(-s_hi), __fsub_rn(1.0f, s_lo));
}

__device__ __forceinline__ float hazard_lognormal(const LawF& L, float tau)
{
    if (!(tau > 0.0f))
        return 0.0f;
    float zh, zl;
    lognormal_z(L, tau, zh, zl);
    if (zh < -2.0f) {
        const float ez = exp_neg_z2(zh, zl);
        const float erfc_z = __fsub_rn(2.0f, erfcf(-zh));
        return __fdiv_rn(__fmul_rn(L.p2, ez), __fmul_rn(tau, erfc_z));
    }
    return __fdiv_rn(L.p2, __fmul_rn(tau, erfcxf(zh)));
}

__device__ __forceinline__ float hazard(const LawF& L, float tau)
{
    switch (L.kind) {
    case kLawExp:
        return L.p0;
    case kLawLogNormal:
        return hazard_lognormal(L, tau);
    case kLawWeibull:
        // h = (k/s) (tau/s)^(k-1); powf(0, 0) = 1 gives h(0) = 1/s for k = 1
        return __fmul_rn(L.p0, powf(__fmul_rn(tau, L.p1), L.p2));
    case kLawErlang: {
        // h = r (r tau)^(k-1)/(k-1)! / sum_{n<k} (r tau)^n / n!
        const float r = L.p0;
        const float x = __fmul_rn(r, tau);
        if (x <= 1.0f) {
            float t = 1.0f, s = 1.0f;
            for (int n = 1; n < L.k; ++n) {
                t = __fmul_rn(t, __fdiv_rn(x, (float)n));
                s = __fadd_rn(s, t);
            }
            return __fdiv_rn(__fmul_rn(r, t), s);
        }
        // same ratio divided through by x^(k-1)/(k-1)!: r / sum_j (k-1)!/(k-1-j)! x^-j
        const float y = __fdiv_rn(1.0f, x);
        float s = 1.0f;
        for (int m = 1; m < L.k; ++m)
            s = __fadd_rn(1.0f, __fmul_rn(__fmul_rn((float)m, y), s));
        return __fdiv_rn(r, s);
    }
    default:
        return 0.0f;
    }
}

// Probability densities in FP32 (shedding profiles, Section 5.3), from the
// textbook definitions:
//   EXP        f = r e^{-r tau}
//   LOGNORMAL  f = e^{-z^2} / (tau sigma sqrt(2 pi)), z as in the hazard
//              (1 / (sigma sqrt(2 pi)) = p2 / 2)
//   WEIBULL    f = (k/s) x^(k-1) e^{-x^k}, x = tau / s
//   ERLANG     f = r (r tau)^(k-1) / (k-1)! e^{-r tau}
__device__ __forceinline__ float density(const LawF& L, float tau)
{
    if (!(tau >= 0.0f))
        return 0.0f;
    switch (L.kind) {
    case kLawExp:
        return __fmul_rn(L.p0, expf(-__fmul_rn(L.p0, tau)));
    case kLawLogNormal: {
        if (!(tau > 0.0f))
            return 0.0f;
        float zh, zl;
        lognormal_z(L, tau, zh, zl);
        return __fdiv_rn(__fmul_rn(__fmul_rn(0.5f, L.p2), exp_neg_z2(zh, zl)), tau);
    }
    case kLawWeibull: {
        const float x = __fmul_rn(tau, L.p1);
        const float xk1 = powf(x, L.p2);                   // x^(k-1); powf(0, 0) = 1
        return __fmul_rn(__fmul_rn(L.p0, xk1), expf(-__fmul_rn(xk1, x)));
    }
    case kLawErlang: {
        const float r = L.p0;
        const float x = __fmul_rn(r, tau);
        float t = 1.0f;
        for (int n = 1; n < L.k; ++n)
            t = __fmul_rn(t, __fdiv_rn(x, (float)n));
        return __fmul_rn(__fmul_rn(r, t), expf(-x));
    }
    default:
        return 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Age storage: FP32 math, round-to-nearest-even on the store (Section 5.7).
// ---------------------------------------------------------------------------
template <typename AgeT> struct AgeIO;
template <> struct AgeIO<float> {
    static __device__ __forceinline__ float load(float v) { return v; }
    static __device__ __forceinline__ float store(float v) { return v; }
};
template <> struct AgeIO<__half> {
    static __device__ __forceinline__ float load(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half store(float v) { return __float2half_rn(v); }
};
template <> struct AgeIO<__nv_bfloat16> {
    static __device__ __forceinline__ float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 store(float v) { return __float2bfloat16_rn(v); }
};

// Bernoulli probability of a rate over the step: p = 1 - exp(-lambda dt)
__device__ __forceinline__ float p_of_rate(const ModelF& M, float lambda)
{
    return lambda > 0.0f ? -expm1f(-__fmul_rn(lambda, M.dt)) : 0.0f;
}

// the same with the step's own size (adaptive step)
__device__ __forceinline__ float p_of_rate_dt(float lambda, float dt)
{
    return lambda > 0.0f ? -expm1f(-__fmul_rn(lambda, dt)) : 0.0f;
}

// the age after one more step in storage: one FP32 add, round to storage
__device__ __forceinline__ float age_step_stored(float age, float dt, int age_dtype)
{
    const float v = __fadd_rn(age, dt);
    if (age_dtype == kAgeF16)
        return __half2float(__float2half_rn(v));
    if (age_dtype == kAgeBF16)
        return __bfloat162float(__float2bfloat16_rn(v));
    return v;
}

// beta s(tau) of the source-node infectivity (Eq. 8): s = the hazard
// (mode 1) or the density (mode 2) of the shedding law
__device__ __forceinline__ float shed_value(const LawF& L, int mode, float beta, float tau)
{
    const float s = mode == 1 ? hazard(L, tau) : density(L, tau);
    return __fmul_rn(beta, s);
}

// Bounds checks of bounds-checked builds (FS_DEBUG_BOUNDS): an index at or
// beyond its bound records kErrBounds with the index and the check's site in
// the control block (the first one wins) and the access it guards is skipped.
// Other builds compile every check to `true`.
static __device__ __noinline__ bool bounds_reject(DevCtl* ctl, int site, long long idx)
{
    if (atomicCAS(&ctl->error, 0, kErrBounds) == 0) {
        ctl->dbg_index = idx;
        ctl->dbg_site = site;
    }
    return false;
}
#ifdef FS_DEBUG_BOUNDS
#define FS_IN_BOUNDS(ctl, site, idx, bound) \
    ((unsigned long long)(long long)(idx) < (unsigned long long)(long long)(bound) \
         ? true                                                                         \
         : ::fs::bounds_reject((ctl), (site), (long long)(idx)))
#else
#define FS_IN_BOUNDS(ctl, site, idx, bound) true
#endif

// Adds one warp's step totals into its delta slot of row j (every lane of the
// warp calls this with its own counts; lanes 0..3 issue one atomic each, and
// only for non-zero totals). No barrier: warps that finish early leave.
__device__ __forceinline__ void warp_add_deltas(unsigned long long* deltas, int j, uint32_t fS, uint32_t fE,
                                                uint32_t fI, unsigned long long dS)
{
    fS = __reduce_add_sync(0xffffffffu, fS);
    fE = __reduce_add_sync(0xffffffffu, fE);
    fI = __reduce_add_sync(0xffffffffu, fI);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        dS += __shfl_xor_sync(0xffffffffu, dS, o);
    const int lane = threadIdx.x & 31;
    if (lane < kDeltaFields) {
        const unsigned long long v = lane == 0 ? fS : lane == 1 ? fE : lane == 2 ? fI : dS;
        if (v) {
            const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
            atomicAdd(deltas + (int64_t)j * kDeltaRow + (w & (kDeltaSlots - 1)) * kDeltaFields + lane, v);
        }
    }
}

// Memoised probability of an E/I node of age `age` from slot 1 of its law's
// two-slot table row (age0, p0, age1, p1); slot 0 is read by the caller as 8
// bytes and this is called only when slot 0 holds another age. Returns -1
// when slot 1 does not hold `age` either.
__device__ __forceinline__ float ptab_slot1(const float4* row, float age)
{
    const float2 e1 = __ldg(reinterpret_cast<const float2*>(row) + 1);
    return e1.x == age ? e1.y : -1.0f;
}

struct TailResult {
    int x;        // new compartment
    float age;    // new age (FP32 value, rounded on store by the caller)
    bool fired;
};

// Bounded wait on an mbarrier phase (TMA completion). Returns false when the
// iteration limit runs out; the caller records an error and skips the data.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar_smem, uint32_t phase, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar_smem), "r"(phase)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

}  // namespace fs
