// fs_push.cu -- the fused renewal step (FlashSpread, arXiv 2604.22092,
// Algorithm 3 at a fixed step) with the infection pressure of S nodes kept up
// to date by pushes instead of being recounted by a gather every step.
//
// With unit weights and constant shedding (Eq. 3 with s = 1), the pressure
// on an S node i is beta times c_i, the number of its in-neighbours in I.
// The gather form recounts c_i for every S node at every step, although c_i
// only changes when an in-neighbour enters or leaves I, which each node does
// at most once per epidemic. Here each node keeps c_i; a node that enters I
// adds 1 to the count of every node whose row lists it (the transposed CSR,
// built once per graph), and a node that leaves I subtracts 1. Counts are
// integers, so they equal the gathered counts exactly, in any order.
//
// One launch per step stays race-free: counts are read during step k while
// the pushes made during step k must only be seen from step k + 1 on. Pushes
// therefore go to a pending word of parity k & 1; during step k an S node
// adds the pending word of parity (k - 1) & 1 (the pushes of step k - 1)
// into its count and clears it, and no thread pushes into that parity during
// step k. A pending word holds separate +1 and -1 tallies so that atomic
// adds never borrow across fields:
//   thread class (in-degree <= 255): count u8; pending u16 per node, +1
//     tally in the low byte, -1 tally in the high byte, added through the
//     32-bit word that holds it;
//   merge class: count u32; pending u64, +1 tally in the low 32 bits, -1
//     tally in the high 32 bits.
// A tally never exceeds the node's in-degree: S nodes clear theirs every
// step, and any node receives at most one +1 and one -1 per in-neighbour
// over a whole run.
//
// The step itself (probability, Philox draw, transition, renewal age,
// counts) is the same code as the gather form's (fs_device.cuh), so results
// are identical to it bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "fs_device.cuh"
#include "fs_launch.h"

namespace fs {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

// the hazard of an E or I node (adaptive step: evaluated every step; out of line)
__device__ __noinline__ float rate_ei(const ModelF& M, int x, float age)
{
    return hazard(x == kE ? M.lat : M.inf, age);
}


// an E/I probability whose table slot 0 holds another age: slot 1, else
// direct evaluation (rare; out of line)
__device__ __noinline__ float p_table_miss(const StepArgs& a, int x, float age)
{
    const int n = __float2int_rn(__fmul_rn(age, a.M.inv_dt));
    if ((unsigned)n < (unsigned)kPTableN) {
        const float p1 = ptab_slot1(a.ptab + (x == kI ? kPTableN : 0) + n, age);
        if (p1 >= 0.0f)
            return p1;
    }
    return p_of_rate(a.M, hazard(x == kE ? a.M.lat : a.M.inf, age));
}

struct PushDeltas {
    uint32_t fS = 0, fE = 0, fI = 0, dS = 0;
};

// successor compartment and renewal age of one node after its decision
__device__ __forceinline__ int next_state(const StepArgs& a, int x, bool fired)
{
    if (!fired)
        return x;
    return (x == kS) ? (a.M.model == kSEIR ? kE : kI) : (x + 1);
}

// eight ages of storage type AgeT as FP32 values
template <typename AgeT> struct AgeVec8;
template <> struct AgeVec8<float> {
    // the 32 bytes of eight ages as two 16-byte words (loaded ahead of use)
    static __device__ __forceinline__ void raw(const float* p, uint4& r0, uint4& r1)
    {
        r0 = *reinterpret_cast<const uint4*>(p);
        r1 = *reinterpret_cast<const uint4*>(p + 4);
    }
    static __device__ __forceinline__ void from_raw(uint4 r0, uint4 r1, float (&f)[8])
    {
        f[0] = __uint_as_float(r0.x); f[1] = __uint_as_float(r0.y);
        f[2] = __uint_as_float(r0.z); f[3] = __uint_as_float(r0.w);
        f[4] = __uint_as_float(r1.x); f[5] = __uint_as_float(r1.y);
        f[6] = __uint_as_float(r1.z); f[7] = __uint_as_float(r1.w);
    }
    static __device__ __forceinline__ void load(const float* p, float (&f)[8])
    {
        const float4 v0 = *reinterpret_cast<const float4*>(p), v1 = *reinterpret_cast<const float4*>(p + 4);
        f[0] = v0.x; f[1] = v0.y; f[2] = v0.z; f[3] = v0.w;
        f[4] = v1.x; f[5] = v1.y; f[6] = v1.z; f[7] = v1.w;
    }
    static __device__ __forceinline__ void store(float* p, const float (&f)[8])
    {
        *reinterpret_cast<float4*>(p) = make_float4(f[0], f[1], f[2], f[3]);
        *reinterpret_cast<float4*>(p + 4) = make_float4(f[4], f[5], f[6], f[7]);
    }
};
__device__ __forceinline__ __half bits_to(const __half*, unsigned short b) { return __ushort_as_half(b); }
__device__ __forceinline__ __nv_bfloat16 bits_to(const __nv_bfloat16*, unsigned short b)
{
    return __ushort_as_bfloat16(b);
}
__device__ __forceinline__ unsigned short to_bits(__half h) { return __half_as_ushort(h); }
__device__ __forceinline__ unsigned short to_bits(__nv_bfloat16 h) { return __bfloat16_as_ushort(h); }

template <typename H> struct AgeVec8Half {
    static __device__ __forceinline__ void raw(const H* p, uint4& r0, uint4& r1)
    {
        r0 = *reinterpret_cast<const uint4*>(p);
        r1 = make_uint4(0u, 0u, 0u, 0u);
    }
    static __device__ __forceinline__ void from_raw(uint4 v, uint4, float (&f)[8])
    {
        const H* tag = nullptr;
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            f[2 * q] = AgeIO<H>::load(bits_to(tag, (unsigned short)(w[q] & 0xffffu)));
            f[2 * q + 1] = AgeIO<H>::load(bits_to(tag, (unsigned short)(w[q] >> 16)));
        }
    }
    static __device__ __forceinline__ void load(const H* p, float (&f)[8])
    {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        from_raw(v, v, f);
    }
    static __device__ __forceinline__ void store(H* p, const float (&f)[8])
    {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            w[q] = (uint32_t)to_bits(AgeIO<H>::store(f[2 * q])) |
                   ((uint32_t)to_bits(AgeIO<H>::store(f[2 * q + 1])) << 16);
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};
template <> struct AgeVec8<__half> : AgeVec8Half<__half> {};
template <> struct AgeVec8<__nv_bfloat16> : AgeVec8Half<__nv_bfloat16> {};

__device__ __forceinline__ uint32_t byte_of(uint2 v, int u)
{
    return ((u < 4 ? v.x : v.y) >> (8 * (u & 3))) & 0xffu;
}

__device__ __forceinline__ void set_byte(uint2& v, int u, uint32_t b)
{
    const uint32_t sh = 8 * (u & 3), m = ~(0xffu << sh);
    if (u < 4)
        v.x = (v.x & m) | (b << sh);
    else
        v.y = (v.y & m) | (b << sh);
}

// ---------------------------------------------------------------------------
// One round of a warp: every lane holds one item, a group of kPushG
// consecutive thread-class nodes or one merge-class node. The nodes that can
// change this step (E and I nodes, S nodes with an infectious in-neighbour)
// are queued in shared memory and the 32 lanes share the queue evenly, so a
// round costs a table lookup and a Philox draw per queued node and a few
// byte-parallel (SWAR) operations per group: classification, the fold of the
// pending tallies and the transitions work on eight nodes at once.
// ---------------------------------------------------------------------------
constexpr int kWarpSlots = 32 * kPushG;       // node slots of a round: lane * kPushG + u
// queued nodes a lane draws for at once (2 measured faster than 3 or 4,
// which need more registers than the 64 a thread has)
constexpr int kDrawsPerPass = 2;

struct WarpScratch {
    uint8_t xb[kWarpSlots];       // state of the node in each slot (R for empty slots)
    uint8_t cb[kWarpSlots];       // infectious in-neighbour count (thread class)
    uint8_t fb[kWarpSlots];       // decision: 0xff fired, 0 not
    uint8_t q[kWarpSlots];        // the round's queue of slots that draw
    float age[kWarpSlots];        // age of the E/I node in each slot
    int32_t base[32];             // first node of each lane's item
    uint32_t hc[32];              // count of a lane's merge-class node, ~0 for a group
    uint32_t ev[kWarpSlots + 32]; // deferred push events: node | (1u << 31) when it left I
};

enum { kItemNone = 0, kItemGroup = 1, kItemHub = 2 };

// The loads of a group that can be issued before it is processed (a round
// ahead): its states and, while many nodes are S, its counts and pending
// tallies. Every word read belongs to this thread's group, so no other thread
// writes it during the step.
struct GroupLoads {
    uint2 xs;
    uint2 c8;
    uint4 pd;
    bool have_cp;        // c8 and pd loaded
};

// The ages of a group loaded together with its states while E and I nodes
// are common (raw storage words; ag1 unused for 16-bit ages)
struct GroupAges {
    uint4 ag0, ag1;
    bool have;
};

__device__ __forceinline__ GroupLoads group_loads(const StepArgs& a, uint32_t par, int64_t t, int64_t n_grp,
                                                  bool spec_s)
{
    GroupLoads g;
    g.xs = make_uint2(0x03030303u, 0x03030303u);
    g.c8 = make_uint2(0u, 0u);
    g.pd = make_uint4(0u, 0u, 0u, 0u);
    g.have_cp = false;
    if (t < n_grp && FS_IN_BOUNDS(a.ctl, kSiteGroup, t * kPushG + kPushG - 1, a.x_len)) {
        const int i0 = (int)(t * kPushG);
        g.xs = *reinterpret_cast<const uint2*>(a.X + i0);
        if (spec_s) {
            g.c8 = *reinterpret_cast<const uint2*>(a.cnt8 + i0);
            g.pd = *reinterpret_cast<const uint4*>(a.pd16[par ^ 1u] + i0);
            g.have_cp = true;
        }
    }
    return g;
}

// ages of a whole group (thread class, every node below n_thr) when spec_ei
template <typename AgeT>
__device__ __forceinline__ GroupAges group_ages(const StepArgs& a, int64_t t, int64_t n_grp, bool spec_ei)
{
    GroupAges g;
    g.ag0 = make_uint4(0u, 0u, 0u, 0u);
    g.ag1 = g.ag0;
    g.have = false;
    if (spec_ei && t < n_grp && (t + 1) * kPushG <= (int64_t)a.n_thr &&
        FS_IN_BOUNDS(a.ctl, kSiteGroup, t * kPushG + kPushG - 1, a.x_len)) {
        AgeVec8<AgeT>::raw(static_cast<const AgeT*>(a.A) + t * kPushG, g.ag0, g.ag1);
        g.have = true;
    }
    return g;
}

// states of a group with the bytes of nodes at or beyond n_thr (a partial
// last group) set to R
__device__ __forceinline__ uint2 group_states(const StepArgs& a, int i0, uint2 xs)
{
    const int nv = a.n_thr - i0;
    if (nv < kPushG) {
#pragma unroll
        for (int u = 0; u < kPushG; ++u)
            if (u >= nv)
                set_byte(xs, u, kR);
    }
    return xs;
}

// A group in which nothing can happen this step: no E or I node, and every S
// node with count 0 and no pending push (R nodes' tallies are never read).
// Its nodes draw nothing and keep their state, so the step skips it. Needs
// the counts and tallies when the group has an S node.
__device__ __forceinline__ bool group_idle(const StepArgs& a, uint32_t par, int64_t t, int64_t n_grp,
                                           GroupLoads& gl)
{
    if (t >= n_grp)
        return true;
    const int i0 = (int)(t * kPushG);
    const uint2 xs = group_states(a, i0, gl.xs);
    const uint32_t ei = __vcmpeq4(xs.x, 0x01010101u) | __vcmpeq4(xs.x, 0x02020202u) |
                        __vcmpeq4(xs.y, 0x01010101u) | __vcmpeq4(xs.y, 0x02020202u);
    if (ei)
        return false;
    const uint32_t sx = __vcmpeq4(xs.x, 0u), sy = __vcmpeq4(xs.y, 0u);   // 0xff per S byte
    if ((sx | sy) == 0u)
        return true;                               // R only
    if (!gl.have_cp) {
        gl.c8 = *reinterpret_cast<const uint2*>(a.cnt8 + i0);
        gl.pd = *reinterpret_cast<const uint4*>(a.pd16[par ^ 1u] + i0);
        gl.have_cp = true;
    }
    // S-byte masks spread to the 16-bit tally fields
    const uint32_t m0 = __byte_perm(sx, 0u, 0x1100u), m1 = __byte_perm(sx, 0u, 0x3322u);
    const uint32_t m2 = __byte_perm(sy, 0u, 0x1100u), m3 = __byte_perm(sy, 0u, 0x3322u);
    return ((gl.c8.x & sx) | (gl.c8.y & sy) | (gl.pd.x & m0) | (gl.pd.y & m1) | (gl.pd.z & m2) |
            (gl.pd.w & m3)) == 0u;
}

// bit u of the result = top bit of byte u (bytes of a __vcmpeq4-style mask:
// 0x00 or 0xff), for the four bytes of a word
__device__ __forceinline__ uint32_t byte_mask_bits(uint32_t m)
{
    return ((m & 0x01010101u) * 0x01020408u) >> 24;
}

__device__ __forceinline__ uint32_t byte_mask_bits(uint2 m)
{
    return byte_mask_bits(m.x) | (byte_mask_bits(m.y) << 4);
}

__device__ __forceinline__ uint2 vcmpeq(uint2 v, uint32_t b)
{
    return make_uint2(__vcmpeq4(v.x, b), __vcmpeq4(v.y, b));
}

__device__ __forceinline__ uint2 operator|(uint2 p, uint2 q) { return make_uint2(p.x | q.x, p.y | q.y); }
__device__ __forceinline__ uint2 operator&(uint2 p, uint2 q) { return make_uint2(p.x & q.x, p.y & q.y); }
__device__ __forceinline__ uint2 operator~(uint2 p) { return make_uint2(~p.x, ~p.y); }

// Bernoulli probability (and, with ADAPTIVE, the rate into lmax) of a queued
// node: state x, count c (S), age (E/I)
template <bool ADAPTIVE>
__device__ __forceinline__ float queued_p(const StepArgs& a, int x, uint32_t c, float age, float dt, float& lmax)
{
    if constexpr (ADAPTIVE) {
        const float lam = x == kS ? __fmul_rn(a.M.beta, (float)c) : rate_ei(a.M, x, age);
        lmax = fmaxf(lmax, lam);
        return p_of_rate_dt(lam, dt);
    } else {
        if (x == kS)
            return c < (uint32_t)kPSTableN ? __ldg(a.ps + c) : p_of_rate(a.M, __fmul_rn(a.M.beta, (float)c));
        const int n = __float2int_rn(__fmul_rn(age, a.M.inv_dt));
        float2 e = make_float2(-1.0f, 0.0f);                  // no entry: never equals an age
        if ((unsigned)n < (unsigned)kPTableN)
            e = __ldg(reinterpret_cast<const float2*>(a.ptab + (x == kI ? kPTableN : 0) + n));
        return e.x == age ? e.y : p_table_miss(a, x, age);    // slot 1, else direct evaluation
    }
}

// +1 / -1 into the pending tally of node j (parity par)
__device__ __forceinline__ void push_pending(const StepArgs& a, uint32_t par, uint32_t j, bool minus)
{
    if (j < (uint32_t)a.n_thr) {
        unsigned int* w = reinterpret_cast<unsigned int*>(a.pd16[par]) + (j >> 1);
        atomicAdd(w, (minus ? 0x100u : 0x1u) << ((j & 1u) << 4));
    } else if (j < (uint32_t)a.n) {
        atomicAdd(a.pd64[par] + (j - (uint32_t)a.n_thr), minus ? (1ull << 32) : 1ull);
    } else {
        (void)FS_IN_BOUNDS(a.ctl, kSitePushTarget, j, a.n);
    }
}

// +1 straight into the count of node j (initial counts)
__device__ __forceinline__ void push_count(const StepArgs& a, uint32_t j)
{
    if (j < (uint32_t)a.n_thr)
        atomicAdd(reinterpret_cast<unsigned int*>(a.cnt8) + (j >> 2), 1u << ((j & 3u) << 3));
    else if (j < (uint32_t)a.n)
        atomicAdd(a.hcnt + (j - (uint32_t)a.n_thr), 1u);
    else
        (void)FS_IN_BOUNDS(a.ctl, kSitePushTarget, j, a.n);
}

template <bool INIT>
__device__ __forceinline__ void push_one(const StepArgs& a, uint32_t par, uint32_t j, bool minus)
{
    if constexpr (INIT)
        push_count(a, j);
    else
        push_pending(a, par, j, minus);
}

template <bool INIT>
__device__ __forceinline__ void warp_push(const StepArgs& a, uint32_t par, uint32_t ev, uint32_t neg, int base,
                                          uint32_t* __restrict__ list);
__device__ __forceinline__ void warp_push_defer(const StepArgs& a, uint32_t par, uint32_t ev, uint32_t neg,
                                                int base, uint32_t* __restrict__ list, int& pend);

// One round of the warp (every lane calls this; item t of this lane, t >=
// total for none; gl = the group's early loads). Returns nothing: states,
// ages, counts and tallies are stored, pushes are made, deltas accumulated.
template <typename AgeT, bool ADAPTIVE, bool DEFER>
__device__ __forceinline__ void warp_round(const StepArgs& a, uint32_t par, uint32_t step, int64_t t,
                                           const GroupLoads& gl, const GroupAges& ga, int64_t n_grp, int64_t total,
                                           float dt, float& lmax, PushDeltas& ld, WarpScratch& w, int& pend)
{
    const int lane = threadIdx.x & 31;
    const int slot0 = lane * kPushG;
    int kind = t < n_grp ? kItemGroup : (t < total ? kItemHub : kItemNone);
    if (kind == kItemHub && !FS_IN_BOUNDS(a.ctl, kSiteGroup, a.n_thr + (t - n_grp), a.n))
        kind = kItemNone;
    uint2 xs = make_uint2(0x03030303u, 0x03030303u);   // R for empty slots
    uint2 sM = make_uint2(0u, 0u), eM = sM, iM = sM;    // 0xff per S / E / I byte
    uint32_t need = 0u;                                 // bit u: slot0 + u draws
    bool clear = false;
    uint2 nc = make_uint2(0u, 0u);
    int base = 0;
    uint32_t hcount = ~0u;
    const AgeT* __restrict__ Ain = static_cast<const AgeT*>(a.A);
    if (kind == kItemGroup) {
        base = (int)(t * kPushG);
        xs = group_states(a, base, gl.xs);
        sM = vcmpeq(xs, 0u);
        eM = vcmpeq(xs, 0x01010101u);
        iM = vcmpeq(xs, 0x02020202u);
        const bool anyS = (sM.x | sM.y) != 0u;
        if (anyS) {
            uint2 c8 = gl.c8;
            uint4 pd = gl.pd;
            if (!gl.have_cp) {
                c8 = *reinterpret_cast<const uint2*>(a.cnt8 + base);
                pd = *reinterpret_cast<const uint4*>(a.pd16[par ^ 1u] + base);
            }
            // fold the pending tallies (field u: +1 tally in its low byte, -1
            // tally in its high byte) into the counts, eight at once; an S
            // node's count is in [0, 255], so the byte-wise wrap is exact
            const uint32_t plus0 = __byte_perm(pd.x, pd.y, 0x6420u), minus0 = __byte_perm(pd.x, pd.y, 0x7531u);
            const uint32_t plus1 = __byte_perm(pd.z, pd.w, 0x6420u), minus1 = __byte_perm(pd.z, pd.w, 0x7531u);
            const uint2 f = make_uint2(__vsub4(__vadd4(c8.x, plus0), minus0), __vsub4(__vadd4(c8.y, plus1), minus1));
            nc = (f & sM) | (c8 & ~sM);               // counts of non-S nodes are left as they were
            clear = (pd.x | pd.y | pd.z | pd.w) != 0u;
            need = byte_mask_bits(sM & ~vcmpeq(nc, 0u));
        }
        const uint2 eiM = eM | iM;
        if ((eiM.x | eiM.y) != 0u) {
            need |= byte_mask_bits(eiM);
            float ag[kPushG];
            if (ga.have) {
                AgeVec8<AgeT>::from_raw(ga.ag0, ga.ag1, ag);
            } else if (base + kPushG <= a.n_thr) {
                AgeVec8<AgeT>::load(Ain + base, ag);
            } else {
#pragma unroll
                for (int u = 0; u < kPushG; ++u)
                    ag[u] = base + u < a.n_thr ? AgeIO<AgeT>::load(Ain[base + u]) : 0.0f;
            }
            *reinterpret_cast<float4*>(w.age + slot0) = make_float4(ag[0], ag[1], ag[2], ag[3]);
            *reinterpret_cast<float4*>(w.age + slot0 + 4) = make_float4(ag[4], ag[5], ag[6], ag[7]);
        }
    } else if (kind == kItemHub) {
        base = a.n_thr + (int)(t - n_grp);
        const int x = a.X[base];
        xs.x = 0x03030300u | (uint32_t)x;
        const int r = base - a.n_thr;
        if (x == kS) {
            unsigned long long* pr = a.pd64[par ^ 1u] + r;
            const unsigned long long d = *pr;
            uint32_t c = a.hcnt[r];
            if (d) {
                c = c + (uint32_t)(d & 0xffffffffull) - (uint32_t)(d >> 32);
                a.hcnt[r] = c;
                *pr = 0ull;
            }
            hcount = c;
            need = c != 0u ? 1u : 0u;
        } else if (x == kE || x == kI) {
            w.age[slot0] = AgeIO<AgeT>::load(Ain[base]);
            need = 1u;
        }
    }
    *reinterpret_cast<uint2*>(w.xb + slot0) = xs;
    *reinterpret_cast<uint2*>(w.cb + slot0) = nc;
    *reinterpret_cast<uint2*>(w.fb + slot0) = make_uint2(0u, 0u);
    w.base[lane] = base;
    w.hc[lane] = hcount;
    // the queue: slots that draw, lane by lane
    const uint32_t cnt = (uint32_t)__popc(need);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += y;
    }
    const int total_q = (int)__shfl_sync(kFull, incl, 31);
    {
        int j = (int)(incl - cnt);
        uint32_t m = need;
        while (m) {
            const int u = __ffs(m) - 1;
            m &= m - 1u;
            w.q[j++] = (uint8_t)(slot0 + u);
        }
    }
    __syncwarp();
    // the draws: kDrawsPerPass queued nodes per lane per pass (independent
    // chains of table loads and Philox rounds; a pass's missing entries
    // repeat its first one and store nothing)
    for (int e0 = lane; e0 < total_q; e0 += 32 * kDrawsPerPass) {
        int sl[kDrawsPerPass];
        float pr[kDrawsPerPass], ur[kDrawsPerPass];
        sl[0] = w.q[e0];
#pragma unroll
        for (int d = 1; d < kDrawsPerPass; ++d)
            sl[d] = e0 + 32 * d < total_q ? (int)w.q[e0 + 32 * d] : sl[0];
#pragma unroll
        for (int d = 0; d < kDrawsPerPass; ++d) {
            const int s_ = sl[d];
            const uint32_t h = w.hc[s_ >> 3];
            const uint32_t c = h != ~0u ? h : (uint32_t)w.cb[s_];
            const int node = w.base[s_ >> 3] + (s_ & (kPushG - 1));
            const uint32_t orig = a.perm ? (uint32_t)__ldg(a.perm + node) : (uint32_t)node;
            pr[d] = queued_p<ADAPTIVE>(a, w.xb[s_], c, w.age[s_], dt, lmax);
            ur[d] = uniform24(a.M.key0, a.M.key1, a.M.rep, step, orig);
        }
#pragma unroll
        for (int d = 0; d < kDrawsPerPass; ++d)
            if (d == 0 || e0 + 32 * d < total_q)
                w.fb[sl[d]] = ur[d] < pr[d] ? 0xffu : 0u;
    }
    __syncwarp();
    // transitions, renewal ages, in-place stores, push events and deltas
    uint32_t ev = 0u, neg = 0u;
    if (kind == kItemGroup) {
        const uint2 F = *reinterpret_cast<const uint2*>(w.fb + slot0);
        if ((F.x | F.y) != 0u) {
            // SEIR: every firing node moves to the next compartment (+1);
            // SIR: S -> I is +2, I -> R is +1
            uint2 inc = F & make_uint2(0x01010101u, 0x01010101u);
            if (a.M.model != kSEIR)
                inc = make_uint2(inc.x + (F.x & sM.x & 0x01010101u), inc.y + (F.y & sM.y & 0x01010101u));
            const uint2 nx = make_uint2(xs.x + inc.x, xs.y + inc.y);     // no byte carries: R never fires
            const uint2 enterI = F & (a.M.model == kSEIR ? eM : sM);
            ev = byte_mask_bits(enterI | (F & iM));
            neg = byte_mask_bits(F & iM);
            ld.fS += (uint32_t)(__popc((F & sM).x) + __popc((F & sM).y)) >> 3;
            ld.fE += (uint32_t)(__popc((F & eM).x) + __popc((F & eM).y)) >> 3;
            ld.fI += (uint32_t)(__popc((F & iM).x) + __popc((F & iM).y)) >> 3;
            uint32_t fs_bits = byte_mask_bits(F & sM);
            while (fs_bits) {
                const int u = __ffs(fs_bits) - 1;
                fs_bits &= fs_bits - 1u;
                ld.dS += (uint32_t)__ldg(a.deg + base + u);
            }
            if (base + kPushG <= a.n_thr) {
                *reinterpret_cast<uint2*>(a.X + base) = nx;
            } else {
#pragma unroll
                for (int u = 0; u < kPushG; ++u)
                    if (base + u < a.n_thr && byte_of(nx, u) != byte_of(xs, u))
                        a.X[base + u] = (uint8_t)byte_of(nx, u);
            }
        }
        const uint2 eiM = eM | iM;
        if ((eiM.x | eiM.y) != 0u) {
            // renewal ages: 0 on firing, E/I ages advance by dt (FP32 add,
            // rounded to storage on the store); S/R ages stay 0
            const uint32_t fb = byte_mask_bits(F), eb = byte_mask_bits(eiM);
            float ag[kPushG];
#pragma unroll
            for (int u = 0; u < kPushG; ++u) {
                const float g = w.age[slot0 + u];
                ag[u] = ((fb >> u) & 1u) ? 0.0f : (((eb >> u) & 1u) ? __fadd_rn(g, dt) : 0.0f);
            }
            AgeT* __restrict__ Aout = static_cast<AgeT*>(a.A) + base;
            if (base + kPushG <= a.n_thr) {
                AgeVec8<AgeT>::store(Aout, ag);
            } else {
#pragma unroll
                for (int u = 0; u < kPushG; ++u)
                    if (base + u < a.n_thr)
                        Aout[u] = AgeIO<AgeT>::store(ag[u]);
            }
        }
        // the pending tallies just folded in are cleared for the pushes of
        // the next step; counts and tallies of the thread class are padded
        // to whole groups, so these stores never touch another class
        if (clear) {
            *reinterpret_cast<uint2*>(a.cnt8 + base) = nc;
            *reinterpret_cast<uint4*>(a.pd16[par ^ 1u] + base) = make_uint4(0u, 0u, 0u, 0u);
        }
    } else if (kind == kItemHub) {
        const int x = (int)(xs.x & 0xffu);
        if (x != kR) {
            const bool f = w.fb[slot0] != 0u;
            const int y = next_state(a, x, f);
            if (y != x)
                a.X[base] = (uint8_t)y;
            if (f || x == kE || x == kI)
                static_cast<AgeT*>(a.A)[base] = AgeIO<AgeT>::store(f ? 0.0f : __fadd_rn(w.age[slot0], dt));
            if ((y == kI) != (x == kI)) {
                ev = 1u;
                neg = x == kI ? 1u : 0u;
            }
            if (f) {
                ld.fS += x == kS;
                ld.fE += x == kE;
                ld.fI += x == kI;
                if (x == kS)
                    ld.dS += (uint32_t)__ldg(a.deg + base);
            }
        }
    }
    if constexpr (DEFER)
        warp_push_defer(a, par, ev, neg, base, w.ev, pend);
    else
        warp_push<false>(a, par, ev, neg, base, w.ev);
}

// ---------------------------------------------------------------------------
// Warp-wide pushes. The lanes' push events (bit u of ev: node base + u
// entered I, or left it when bit u of neg is set) are appended to the warp's
// event list; per batch of 32 events lane e reads event e's transposed row
// bounds, a warp scan of the row lengths flattens the batch's edges into one
// index range, and the 32 lanes stride over it, each finding its event by a
// binary search over the lanes' offsets. A batch costs two dependent memory
// round trips however many events it holds, so a warp that sweeps several
// rounds in one step (large graphs) defers its events until a batch is full
// or its sweep ends: a round with a few events then waits for no push at
// all. Pushes made later in the same step are equivalent: they go to the
// tallies of this step's parity, which are read only by the next step.
// Every lane of the warp must call these.
// ---------------------------------------------------------------------------
constexpr int64_t kPushLongRow = 128;    // rows longer than this are pushed one at a time

// appends the lanes' events at list[pend ..]; returns the new length
__device__ __forceinline__ int warp_events_append(uint32_t ev, uint32_t neg, int base, uint32_t* __restrict__ list,
                                                  int pend)
{
    const int lane = threadIdx.x & 31;
    const uint32_t cnt = (uint32_t)__popc(ev);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += y;
    }
    const int nev = (int)__shfl_sync(kFull, incl, 31);
    if (nev) {
        int j = pend + (int)(incl - cnt);
        uint32_t m = ev;
        while (m) {
            const int u = __ffs(m) - 1;
            m &= m - 1u;
            list[j++] = (uint32_t)(base + u) | (((neg >> u) & 1u) << 31);
        }
    }
    return pend + nev;
}

// the pushes of events list[0 .. nproc)
template <bool INIT>
__device__ __forceinline__ void warp_push_events(const StepArgs& a, uint32_t par, const uint32_t* __restrict__ list,
                                                 int nproc)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int c0 = 0; c0 < nproc; c0 += 32) {
        const int e = c0 + lane;
        int64_t lo = 0, len = 0;
        uint32_t evw = 0u;
        if (e < nproc) {
            evw = list[e];
            const int node = (int)(evw & 0x7fffffffu);
            if (FS_IN_BOUNDS(a.ctl, kSiteOutPtr, node, a.n)) {
                lo = __ldg(a.out_ptr + node);
                len = __ldg(a.out_ptr + node + 1) - lo;
            }
        }
        // long rows (hubs) one at a time, the warp striding over each with
        // its column loads issued four ahead; they leave the flattened batch
        uint32_t lng = __ballot_sync(kFull, len > kPushLongRow);
        while (lng) {
            const int l = __ffs(lng) - 1;
            lng &= lng - 1u;
            const int64_t lo_l = __shfl_sync(kFull, lo, l), len_l = __shfl_sync(kFull, len, l);
            const bool minus = (__shfl_sync(kFull, evw, l) >> 31) != 0u;
            const int32_t* __restrict__ col = a.out_col + lo_l;
            int64_t q = lane;
#ifndef FS_DEBUG_BOUNDS
            for (; q + 96 < len_l; q += 128) {
                const uint32_t j0 = (uint32_t)__ldg(col + q), j1 = (uint32_t)__ldg(col + q + 32);
                const uint32_t j2 = (uint32_t)__ldg(col + q + 64), j3 = (uint32_t)__ldg(col + q + 96);
                push_one<INIT>(a, par, j0, minus);
                push_one<INIT>(a, par, j1, minus);
                push_one<INIT>(a, par, j2, minus);
                push_one<INIT>(a, par, j3, minus);
            }
#endif
            for (; q < len_l; q += 32)
                if (FS_IN_BOUNDS(a.ctl, kSiteOutCol, lo_l + q, a.out_nnz - a.dbg_shrink))
                    push_one<INIT>(a, par, (uint32_t)__ldg(col + q), minus);
        }
        if (len > kPushLongRow)
            len = 0;
        int64_t off = len;                          // inclusive scan of the lengths
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, off, o);
            if (lane >= o)
                off += y;
        }
        const int64_t tot = __shfl_sync(kFull, off, 31);
        off -= len;                                 // exclusive
        // warp-uniform trip count: every lane takes part in every shuffle
        for (int64_t q0 = 0; q0 < tot; q0 += 32) {
            const int64_t q = q0 + lane;
            // the lane (event) whose range holds q: largest l with off_l <= q
            int l = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int64_t o = __shfl_sync(kFull, off, l + step);
                if (o <= q)
                    l += step;
            }
            const int64_t lo_l = __shfl_sync(kFull, lo, l);
            const int64_t off_l = __shfl_sync(kFull, off, l);
            const uint32_t ev_l = __shfl_sync(kFull, evw, l);
            if (q < tot && FS_IN_BOUNDS(a.ctl, kSiteOutCol, lo_l + (q - off_l), a.out_nnz - a.dbg_shrink)) {
                const uint32_t j = (uint32_t)__ldg(a.out_col + lo_l + (q - off_l));
                push_one<INIT>(a, par, j, (ev_l >> 31) != 0u);
            }
        }
    }
    __syncwarp();     // the list is rewritten by the warp's next append
}

// all the lanes' events at once (initial counts)
template <bool INIT>
__device__ __forceinline__ void warp_push(const StepArgs& a, uint32_t par, uint32_t ev, uint32_t neg, int base,
                                          uint32_t* __restrict__ list)
{
    const int nev = warp_events_append(ev, neg, base, list, 0);
    if (nev)
        warp_push_events<INIT>(a, par, list, nev);
}

// the step's events: appended, and pushed in whole batches of 32 once at
// least one is full; the rest (fewer than 32) move to the front of the list.
// The list holds pend (< 32) + one round's events (at most kWarpSlots).
__device__ __forceinline__ void warp_push_defer(const StepArgs& a, uint32_t par, uint32_t ev, uint32_t neg,
                                                int base, uint32_t* __restrict__ list, int& pend)
{
    pend = warp_events_append(ev, neg, base, list, pend);
    if (pend < 32)
        return;
    const int full = pend & ~31, rest = pend & 31;
    warp_push_events<false>(a, par, list, full);
    const int lane = threadIdx.x & 31;
    uint32_t v = 0u;
    if (lane < rest)
        v = list[full + lane];
    __syncwarp();
    if (lane < rest)
        list[lane] = v;
    __syncwarp();
    pend = rest;
}

// the events still deferred when the warp's sweep ends
__device__ __forceinline__ void warp_push_drain(const StepArgs& a, uint32_t par, uint32_t* __restrict__ list,
                                                int& pend)
{
    if (pend)
        warp_push_events<false>(a, par, list, pend);
    pend = 0;
}

constexpr int kScanRounds = 3;      // grid-stride rounds whose loads a warp issues together

// The item loops of one step: one item per lane (the grid covers every item
// at once) or kScanRounds grid-stride rounds at a time. LIST: position q of
// the sweep visits the listed item act[q] (q < n_items), else item q; a
// compile-time choice so that the sweep without a list keeps its own register
// allocation.
template <typename AgeT, bool SCAN, bool ADAPTIVE, bool LIST>
__device__ __forceinline__ void push_items(const StepArgs& a, uint32_t par, int64_t k, bool spec_s, bool spec_ei,
                                           float dt, float& lmax, PushDeltas& ld, WarpScratch& w, int& pend,
                                           const int32_t* __restrict__ act, int64_t n_items)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t n_grp = ((int64_t)a.n_thr + kPushG - 1) / kPushG;
    const int64_t total = n_grp + a.n_m;
    const int64_t stride = (int64_t)gridDim.x * kPushThreads;
    // (item numbers fit 31 bits: at most n / kPushG + n_m < 2^31)
    auto item_at = [&](int64_t q) -> int64_t {
        if constexpr (!LIST)
            return q;
        else
            return q < n_items ? (int64_t)__ldg(act + q) : (int64_t)INT32_MAX;
    };
    // One item per lane (the grid covers every item at once): no scan.
    if constexpr (!SCAN) {
        const int64_t t = item_at((int64_t)blockIdx.x * kPushThreads + tid);
        GroupLoads cur = group_loads(a, par, t, n_grp, spec_s);
        const GroupAges ga = group_ages<AgeT>(a, t, n_grp, false);
        const bool idle = (t < n_grp || t >= total) && group_idle(a, par, t, n_grp, cur);
        if (!__all_sync(kFull, idle))
            warp_round<AgeT, ADAPTIVE, false>(a, par, (uint32_t)k, t, cur, ga, n_grp, total, dt, lmax, ld, w, pend);
    }
    // Warps take kScanRounds grid-stride rounds at a time: the loads that tell
    // whether an item has work (states; counts and tallies while S is common)
    // are issued for all of them together, and only the rounds in which some
    // lane of the warp has work are processed, so a mostly idle sweep (the
    // all-S start, the mostly-R tail) waits for memory once per kScanRounds
    // rounds instead of once per round.
    for (int64_t tb = (int64_t)blockIdx.x * kPushThreads + (tid & ~31); SCAN && tb < n_items;
         tb += (int64_t)kScanRounds * stride) {
        uint32_t busy = 0u;
        {
            GroupLoads gl[kScanRounds];
#pragma unroll
            for (int u = 0; u < kScanRounds; ++u)
                gl[u] = group_loads(a, par, item_at(tb + u * stride + lane), n_grp, spec_s);
#pragma unroll
            for (int u = 0; u < kScanRounds; ++u) {
                const int64_t t = item_at(tb + u * stride + lane);
                const bool idle = (t < n_grp || t >= total) && group_idle(a, par, t, n_grp, gl[u]);
                busy |= (idle ? 0u : 1u) << u;
            }
        }
        uint32_t wb = __reduce_or_sync(kFull, busy);
        while (wb) {
            const int u = __ffs(wb) - 1;
            wb &= wb - 1u;
            const int64_t t = item_at(tb + u * stride + lane);
            // reloaded: these lines were read by the scan just above (the
            // ages, while E/I nodes are common, are issued with them)
            const GroupLoads cur = group_loads(a, par, t, n_grp, spec_s);
            const GroupAges ga = group_ages<AgeT>(a, t, n_grp, spec_ei);
            warp_round<AgeT, ADAPTIVE, true>(a, par, (uint32_t)k, t, cur, ga, n_grp, total, dt, lmax, ld, w, pend);
        }
    }
}

// The listed block-scan sweep out of line: it has its own register
// allocation, and the sweep without a list (inlined into the kernel) keeps
// the allocation it has alone. Results come back by value.
struct PushSweepOut {
    PushDeltas ld;
    float lmax;
    int pend;
};

template <typename AgeT, bool SCAN, bool ADAPTIVE>
__device__ __noinline__ PushSweepOut push_items_listed(const StepArgs& a, uint32_t par, int64_t k, bool spec_s,
                                                        bool spec_ei, float dt, WarpScratch* w, int64_t n_items)
{
    PushSweepOut o;
    o.lmax = 0.0f;
    o.pend = 0;
    push_items<AgeT, SCAN, ADAPTIVE, true>(a, par, k, spec_s, spec_ei, dt, o.lmax, o.ld, *w, o.pend, a.act,
                                           n_items);
    return o;
}

// ---------------------------------------------------------------------------
// One whole step: items are groups of kPushG thread-class nodes, then single
// merge-class nodes; warps stride over them (grid-stride). Each warp adds its
// per-step deltas into its slot and leaves (no CTA-wide barrier).
// ---------------------------------------------------------------------------
template <typename AgeT, bool SCAN, bool ADAPTIVE>
__global__ void __launch_bounds__(kPushThreads, kPushCtasPerSm) push_step_kernel(const __grid_constant__ StepArgs a)
{
    __shared__ WarpScratch scratch[kPushThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    WarpScratch& w = scratch[tid >> 5];
    const int64_t k = a.ctl->step + a.j;
    const uint32_t par = (uint32_t)(k & 1);
    // the step's size: fixed, or (Section 5.2) min(dt_max, eps / (lambda* of
    // the previous step + delta)); this step's largest rate goes to lam[k % 3]
    // for the next one, lam[(k + 1) % 3] (read two steps ago) is cleared for
    // the step after it
    float dt = a.M.dt;
    float lmax = 0.0f;
    if constexpr (ADAPTIVE) {
        const float lp = __uint_as_float(a.ctl->lam[(k + 2) % 3]);
        dt = fminf(a.M.dt, __fdiv_rn(a.eps, __fadd_rn(lp, a.delta)));
        if (blockIdx.x == 0 && tid == 0) {
            a.ctl->lam[(k + 1) % 3] = 0u;
            a.dtrec[a.j] = dt;
        }
    }
    // counts and tallies are loaded a round ahead while S nodes are common
    // (counts of the state at the start of this launch sequence)
    const bool spec_s = (int64_t)a.ctl->counts[0] * 16 >= (int64_t)a.n;
    // in the multi-round sweep, ages are loaded with the states while at
    // least a quarter of the nodes are E or I (then about nine groups in ten
    // hold one)
    const bool spec_ei = ((int64_t)a.ctl->counts[1] + (int64_t)a.ctl->counts[2]) * 4 >= (int64_t)a.n;
    PushDeltas ld;
    int pend = 0;             // deferred push events in w.ev
    // active-node compaction (Section 5.6): the items listed by this launch
    // sequence's refresh, or every item
    const int64_t total = ((int64_t)a.n_thr + kPushG - 1) / kPushG + a.n_m;
    const int64_t na = a.act ? (int64_t)a.ctl->n_act : total;
    if constexpr (SCAN) {
        if (na < total) {
            const PushSweepOut o = push_items_listed<AgeT, SCAN, ADAPTIVE>(a, par, k, spec_s, spec_ei, dt, &w, na);
            ld = o.ld;
            lmax = o.lmax;
            pend = o.pend;
        } else {
            push_items<AgeT, SCAN, ADAPTIVE, false>(a, par, k, spec_s, spec_ei, dt, lmax, ld, w, pend, nullptr,
                                                    total);
        }
    } else {
        // one round: both sweeps inline
        if (na < total)
            push_items<AgeT, SCAN, ADAPTIVE, true>(a, par, k, spec_s, spec_ei, dt, lmax, ld, w, pend, a.act, na);
        else
            push_items<AgeT, SCAN, ADAPTIVE, false>(a, par, k, spec_s, spec_ei, dt, lmax, ld, w, pend, nullptr,
                                                    total);
    }
    warp_push_drain(a, par, w.ev, pend);
    if constexpr (ADAPTIVE) {
        // rates are >= 0, so their FP32 bits order as unsigned integers
        const uint32_t m = __reduce_max_sync(kFull, __float_as_uint(lmax));
        if (lane == 0 && m)
            atomicMax(&a.ctl->lam[k % 3], m);
    }
    warp_add_deltas(a.deltas, a.j, ld.fS, ld.fE, ld.fI, ld.dS);
}

// Initial counts (after init or set_state; counts and tallies zeroed): every
// node in I pushes +1 straight into the counts of its out-neighbours.
__global__ void __launch_bounds__(kPushThreads) push_init_kernel(const __grid_constant__ StepArgs a)
{
    __shared__ uint32_t list[kPushThreads];
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t stride = (int64_t)gridDim.x * kPushThreads;
    for (int64_t t0 = (int64_t)blockIdx.x * kPushThreads + (tid & ~31); t0 < a.n; t0 += stride) {
        const int64_t i = t0 + lane;
        const uint32_t ev = (i < a.n && a.X[i] == kI) ? 1u : 0u;
        warp_push<true>(a, 0u, ev, 0u, (int)i, list + (tid & ~31));
    }
}

// ---------------------------------------------------------------------------
// Transposed CSR of a graph in internal ids, from its SELL-32 blocks (thread
// class: row i's entries are t < deg(i) of its lane) and merge-class CSR:
// out_deg[j] = number of rows listing j, then (after a scan) every row i
// appends itself to the out-row of each j it lists. The order inside an
// out-row is unspecified; pushes commute, so it does not matter.
// ---------------------------------------------------------------------------
template <bool FILL>
__global__ void transpose_kernel(const int64_t* __restrict__ sell_off, const int32_t* __restrict__ sell_col,
                                 const int32_t* __restrict__ deg, int n_thr, const int64_t* __restrict__ m_ptr,
                                 const int32_t* __restrict__ m_col, int n_m, int n,
                                 unsigned long long* __restrict__ cursor, int32_t* __restrict__ out_col)
{
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    auto emit = [&](int j, int i) {
        if ((unsigned)j >= (unsigned)n)     // padding (never inside a row)
            return;
        const unsigned long long pos = atomicAdd(cursor + j, 1ull);
        if constexpr (FILL)
            out_col[pos] = i;
    };
    if (gt < n_thr) {
        const int i = (int)gt;
        const int64_t off = sell_off[i >> 5] + (i & 31);
        const int d = deg[i];
        for (int t = 0; t < d; ++t)
            emit(sell_col[off + 32 * (int64_t)t], i);
    } else {
        // merge-class rows: 32 consecutive threads per row, striding over it
        const int64_t w = (gt - n_thr) >> 5;
        const int l = (int)((gt - n_thr) & 31);
        if (w < n_m) {
            const int r = (int)w;
            for (int64_t e = m_ptr[r] + l; e < m_ptr[r + 1]; e += 32)
                emit(m_col[e], n_thr + r);
        }
    }
}

// Active-node compaction refresh (Section 5.6), at the start of a launch
// sequence: lists the items (groups of kPushG thread-class nodes, merge-class
// nodes) that still hold a non-R node. While fewer than half the nodes are R
// it writes "all items" instead. ctl->n_act is 0 on entry (the previous
// epilogue, init or set_state left it so).
__global__ void push_compact_kernel(const __grid_constant__ StepArgs a)
{
    const int64_t n_grp = ((int64_t)a.n_thr + kPushG - 1) / kPushG;
    const int64_t total = n_grp + a.n_m;
    if ((int64_t)a.ctl->counts[3] * 2 < (int64_t)a.n) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            a.ctl->n_act = (unsigned long long)total;
        return;
    }
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < total; t0 += stride) {
        const int64_t t = t0 + lane;
        bool live = false;
        if (t < n_grp) {
            const int i0 = (int)(t * kPushG);
            uint2 xs = *reinterpret_cast<const uint2*>(a.X + i0);
            const int nv = min(kPushG, a.n_thr - i0);
#pragma unroll
            for (int u = 0; u < kPushG; ++u)
                if (u >= nv)
                    set_byte(xs, u, kR);
            live = (xs.x & xs.y) != 0x03030303u;
        } else if (t < total) {
            live = a.X[a.n_thr + (int)(t - n_grp)] != kR;
        }
        const uint32_t b = __ballot_sync(kFull, live);
        if (b) {
            unsigned long long base = 0ull;
            if (lane == 0)
                base = atomicAdd(&a.ctl->n_act, (unsigned long long)__popc(b));
            base = __shfl_sync(kFull, base, 0);
            if (live)
                a.act[base + __popc(b & ((1u << lane) - 1u))] = (int32_t)t;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename AgeT, bool ADAPTIVE>
static cudaError_t launch_push_step_t(const StepArgs& a, cudaStream_t s, int num_sms)
{
    const int64_t items = ((int64_t)a.n_thr + kPushG - 1) / kPushG + a.n_m;
    const int64_t need = (items + kPushThreads - 1) / kPushThreads;
    const int64_t cap = (int64_t)num_sms * kPushCtasPerSm;
    const int grid = (int)std::max<int64_t>(1, std::min(need, cap));
    // one item per lane when the grid covers them all, else the block scan
    if (need <= cap)
        push_step_kernel<AgeT, false, ADAPTIVE><<<grid, kPushThreads, 0, s>>>(a);
    else
        push_step_kernel<AgeT, true, ADAPTIVE><<<grid, kPushThreads, 0, s>>>(a);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_push_step(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms)
{
    switch (age_dtype) {
    case kAgeF16: return launch_push_step_t<__half, false>(a, s, num_sms);
    case kAgeBF16: return launch_push_step_t<__nv_bfloat16, false>(a, s, num_sms);
    default: return launch_push_step_t<float, false>(a, s, num_sms);
    }
}

cudaError_t launch_push_step_adaptive(const StepArgs& a, int age_dtype, cudaStream_t s, int num_sms)
{
    switch (age_dtype) {
    case kAgeF16: return launch_push_step_t<__half, true>(a, s, num_sms);
    case kAgeBF16: return launch_push_step_t<__nv_bfloat16, true>(a, s, num_sms);
    default: return launch_push_step_t<float, true>(a, s, num_sms);
    }
}

cudaError_t launch_push_compact(const StepArgs& a, cudaStream_t s, int num_sms)
{
    const int64_t items = ((int64_t)a.n_thr + kPushG - 1) / kPushG + a.n_m;
    const int64_t need = (items + kPushThreads - 1) / kPushThreads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * 8));
    push_compact_kernel<<<grid, kPushThreads, 0, s>>>(a);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_push_init(const StepArgs& a, cudaStream_t s, int num_sms)
{
    const int64_t need = ((int64_t)a.n + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * 8));
    push_init_kernel<<<grid, kPushThreads, 0, s>>>(a);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_transpose(const int64_t* sell_off, const int32_t* sell_col, const int32_t* deg, int n_thr,
                             const int64_t* m_ptr, const int32_t* m_col, int n_m, int n,
                             unsigned long long* cursor, int32_t* out_col, bool fill, cudaStream_t s)
{
    const int64_t threads = (int64_t)n_thr + (int64_t)n_m * 32;
    if (threads == 0)
        return cudaSuccess;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (fill)
        transpose_kernel<true><<<blocks, 256, 0, s>>>(sell_off, sell_col, deg, n_thr, m_ptr, m_col, n_m, n, cursor,
                                                      out_col);
    else
        transpose_kernel<false><<<blocks, 256, 0, s>>>(sell_off, sell_col, deg, n_thr, m_ptr, m_col, n_m, n, cursor,
                                                       nullptr);
    g_launch_count += 1;
    return cudaGetLastError();
}

}  // namespace fs
