// fs_pack.cu -- packed ensembles: one launch advances every live segment of
// a batch by one step of the fused renewal tau-leap (FlashSpread, arXiv
// 2604.22092, Algorithm 3 at a fixed step), with up to 32 realisations of a
// graph packed node-major so that each column read and each neighbour-mask
// gather serves all of them.
//
// Work items, taken by warps round-robin over the whole grid:
//   * hub rows first (merge-class rows, degree > thread_max_deg): one warp per
//     row; 32 edges per window, each lane loads one neighbour's R-bit mask and
//     one ballot per S replicate counts that replicate's infectious
//     neighbours; lane r then runs replicate r's tail;
//   * SELL items: 32/R_pad nodes of a 32-node slice x R_pad replicates, lane =
//     (node, replicate); lanes of the same node read the same columns
//     (broadcast) and extract their own bit of each neighbour's mask.
// At the start of a launch one warp per segment integrates the previous
// step's per-replicate deltas into the running counts and writes that row of
// the segment's counts output (deltas are double-buffered by local step
// parity, so the integration never races the step that is running).
#include <cuda_runtime.h>

#include <algorithm>

#include "fs_device.cuh"
#include "fs_launch.h"

namespace fs {

namespace {

constexpr uint32_t kFullP = 0xffffffffu;

template <int L> struct MaskOf;
template <> struct MaskOf<8> { using T = uint8_t; };
template <> struct MaskOf<16> { using T = uint16_t; };
template <> struct MaskOf<32> { using T = uint32_t; };

__device__ __noinline__ float pack_p_direct(const ModelF& M, int x, float age)
{
    return p_of_rate(M, hazard(x == kE ? M.lat : M.inf, age));
}

// Bernoulli probability of one (node, replicate), as in the single step
__device__ __forceinline__ float pack_p(const PackScen& S, int x, float age, uint32_t c)
{
    if (x == kS) {
        if (c == 0u)
            return 0.0f;
        if (c < (uint32_t)kPSTableN)
            return __ldg(S.ps + c);
        return p_of_rate(S.M, __fmul_rn(S.M.beta, (float)c));
    }
    if (x == kE || x == kI) {
        const int n = __float2int_rn(__fmul_rn(age, S.M.inv_dt));
        if ((unsigned)n < (unsigned)kPTableN) {
            const float4* row = S.ptab + (x == kI ? kPTableN : 0) + n;
            const float2 e = __ldg(reinterpret_cast<const float2*>(row));
            if (e.x == age)
                return e.y;
            const float p1 = ptab_slot1(row, age);
            if (p1 >= 0.0f)
                return p1;
        }
        return pack_p_direct(S.M, x, age);
    }
    return 0.0f;
}

struct PackTail {
    int x;
    float age;
    bool fired;
};

// the original id is read only when a uniform is drawn (p > 0 implies a
// valid node: padding and absorbed lanes have p = 0)
__device__ __forceinline__ PackTail pack_tail_p(const PackScen& S, int model, int x, float age, float p,
                                                const int32_t* perm, int i, uint32_t step)
{
    bool fired = false;
    if (p > 0.0f) {
        const uint32_t orig = perm ? (uint32_t)__ldg(perm + i) : (uint32_t)i;
        fired = uniform24(S.M.key0, S.M.key1, S.M.rep, step, orig) < p;
    }
    PackTail t;
    if (fired) {
        t.x = (x == kS) ? (model == kSEIR ? kE : kI) : (x + 1);
        t.age = 0.0f;
    } else {
        t.x = x;
        t.age = (x == kE || x == kI) ? __fadd_rn(age, S.M.dt) : 0.0f;
    }
    t.fired = fired;
    return t;
}

__device__ __forceinline__ PackTail pack_tail(const PackScen& S, int model, int x, float age, uint32_t c,
                                              const int32_t* perm, int i, uint32_t step)
{
    return pack_tail_p(S, model, x, age, pack_p(S, x, age, c), perm, i, step);
}

// Adaptive step (Section 5.2) of one replicate: the step's size from the
// largest rate of the previous step (FP32, the single-realisation step's
// operations), and the rate of an E or I replicate (evaluated directly: ages
// leave the fixed-step sequence, so the probability tables do not apply)
__device__ __forceinline__ float pack_dt_of(uint32_t lam_bits, float eps, float delta, float dt_max)
{
    return fminf(dt_max, __fdiv_rn(eps, __fadd_rn(__uint_as_float(lam_bits), delta)));
}

__device__ __noinline__ float pack_rate_ei(const ModelF& M, int x, float age)
{
    return hazard(x == kE ? M.lat : M.inf, age);
}

// pack_tail with the adaptive step of replicate r (segment g.lam != null):
// its rate goes into the step's maximum, its size comes from the previous one
// (s_rate: the rate of an S replicate)
__device__ __forceinline__ PackTail pack_tail_adaptive_rate(const PackSeg& g, int64_t k, int r, int x, float age,
                                                            float s_rate, int i)
{
    const PackScen& S = g.scen[r];
    const float lam = x == kS ? s_rate : ((x == kE || x == kI) ? pack_rate_ei(S.M, x, age) : 0.0f);
    if (lam > 0.0f)
        atomicMax(g.lam + (k % 3) * g.R_pad + r, __float_as_uint(lam));
    const float dt = pack_dt_of(__ldg(g.lam + ((k + 2) % 3) * g.R_pad + r), S.eps, S.delta, S.M.dt);
    const float p = p_of_rate_dt(lam, dt);
    bool fired = false;
    if (p > 0.0f) {
        const uint32_t orig = g.perm ? (uint32_t)__ldg(g.perm + i) : (uint32_t)i;
        fired = uniform24(S.M.key0, S.M.key1, S.M.rep, (uint32_t)k, orig) < p;
    }
    PackTail t;
    if (fired) {
        t.x = (x == kS) ? (g.model == kSEIR ? kE : kI) : (x + 1);
        t.age = 0.0f;
    } else {
        t.x = x;
        t.age = (x == kE || x == kI) ? __fadd_rn(age, dt) : 0.0f;
    }
    t.fired = fired;
    return t;
}

__device__ __forceinline__ PackTail pack_tail_adaptive(const PackSeg& g, int64_t k, int r, int x, float age,
                                                       uint32_t c, int i)
{
    return pack_tail_adaptive_rate(g, k, r, x, age, c ? __fmul_rn(g.scen[r].M.beta, (float)c) : 0.0f, i);
}

// beta s(tau) of an I replicate of new age `age` (FP32, before storage
// rounding) under its scenario's shedding profile (Section 5.3, Eq. 8): the
// age as stored, looked up in the scenario's memoised table when it lies on
// the fixed-step sequence, else evaluated (the single-realisation step's
// operations, so the stored bits are the same)
__device__ __noinline__ float pack_shed_direct(const PackScen& S, float tau)
{
    return shed_value(S.shed, S.shed_mode, S.M.beta, tau);
}

template <typename AgeT>
__device__ __forceinline__ float pack_rho_of(const PackScen& S, float age)
{
    const float a = AgeIO<AgeT>::load(AgeIO<AgeT>::store(age));
    const int n = __float2int_rn(__fmul_rn(a, S.M.inv_dt));
    if ((unsigned)n < (unsigned)kPTableN) {
        const float4* row = S.rtab + n;
        const float2 e = __ldg(reinterpret_cast<const float2*>(row));
        if (e.x == a)
            return e.y;
        const float r1 = ptab_slot1(row, a);
        if (r1 >= 0.0f)
            return r1;
    }
    return pack_shed_direct(S, a);
}

// per-replicate transitions of this step: [S->, E->I, I->R]
__device__ __forceinline__ void add_deltas(const PackSeg& g, int64_t k, int r, uint32_t dS, uint32_t dE,
                                           uint32_t dI)
{
    unsigned long long* d = g.deltas + ((k & 1) * g.R_pad + r) * 3;
    if (dS) atomicAdd(d + 0, (unsigned long long)dS);
    if (dE) atomicAdd(d + 1, (unsigned long long)dE);
    if (dI) atomicAdd(d + 2, (unsigned long long)dI);
}

// Ages of 8 consecutive replicates of one node, as one or two 16-byte loads
template <typename AgeT> struct AgeVec8;
template <> struct AgeVec8<float> {
    float v[8];
    __device__ __forceinline__ void load(const float* p)
    {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    __device__ __forceinline__ void store(float* p) const
    {
        reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
};
template <typename H> struct AgeVec8H {
    float v[8];
    __device__ __forceinline__ void load(const H* p)
    {
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            H lo, hi;
            const uint16_t l16 = (uint16_t)(w[q] & 0xffffu), h16 = (uint16_t)(w[q] >> 16);
            memcpy(&lo, &l16, 2);
            memcpy(&hi, &h16, 2);
            v[2 * q] = AgeIO<H>::load(lo);
            v[2 * q + 1] = AgeIO<H>::load(hi);
        }
    }
    __device__ __forceinline__ void store(H* p) const
    {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const H lo = AgeIO<H>::store(v[2 * q]), hi = AgeIO<H>::store(v[2 * q + 1]);
            uint16_t l16, h16;
            memcpy(&l16, &lo, 2);
            memcpy(&h16, &hi, 2);
            w[q] = (uint32_t)l16 | ((uint32_t)h16 << 16);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};
template <> struct AgeVec8<__half> : AgeVec8H<__half> {};
template <> struct AgeVec8<__nv_bfloat16> : AgeVec8H<__nv_bfloat16> {};

// true when any byte of v equals b (b < 128)
__device__ __forceinline__ bool has_byte(uint64_t v, uint32_t b)
{
    const uint64_t x = v ^ (0x0101010101010101ull * b);
    return ((x - 0x0101010101010101ull) & ~x & 0x8080808080808080ull) != 0ull;
}

// 0xff in every byte of v that is 0 (an S replicate)
__device__ __forceinline__ uint64_t s_bytes(uint64_t v)
{
    return (uint64_t)__vcmpeq4((uint32_t)v, 0u) | ((uint64_t)__vcmpeq4((uint32_t)(v >> 32), 0u) << 32);
}

// bit r of b (r < 4) -> 1 << (16 r): one 16-bit tally field per replicate
__device__ __forceinline__ uint64_t spread16(uint32_t b)
{
    return (uint64_t)(b & 1u) | ((uint64_t)((b >> 1) & 1u) << 16) | ((uint64_t)((b >> 2) & 1u) << 32) |
           ((uint64_t)((b >> 3) & 1u) << 48);
}

// One out-edge of a packed push: node j receives +1 for each replicate in
// `en` and -1 for each in `lv` (RP-bit masks) in its pending tallies of
// parity par. Thread-class nodes take one 64-bit atomic per 4-replicate word
// holding an event (tallies are bytes inside 16-bit fields and never exceed
// the in-degree, so no carry crosses a field); merge-class nodes one atomic
// per replicate.
template <int RP>
__device__ __forceinline__ void pack_push_edge(const PackSeg& g, uint32_t par, uint32_t j, uint32_t en, uint32_t lv)
{
    if (j < (uint32_t)g.n_thr) {
        unsigned long long* w = reinterpret_cast<unsigned long long*>(g.ppd[par] + (int64_t)j * RP);
#pragma unroll
        for (int q = 0; q < RP / 4; ++q) {
            const uint32_t e4 = (en >> (4 * q)) & 0xfu, l4 = (lv >> (4 * q)) & 0xfu;
            if (e4 | l4)
                atomicAdd(w + q, (unsigned long long)(spread16(e4) | (spread16(l4) << 8)));
        }
    } else if (j < (uint32_t)g.n) {
        unsigned long long* w = g.phpd[par] + (int64_t)(j - (uint32_t)g.n_thr) * RP;
        uint32_t m = en | lv;
        while (m) {
            const int r = __ffs(m) - 1;
            m &= m - 1u;
            atomicAdd(w + r, ((en >> r) & 1u) ? 1ull : (1ull << 32));
        }
    }
}

// Warp-wide packed pushes: lane l's event is node `node` with replicate masks
// (en, lv) (both 0: no event). The warp flattens the events' transposed rows
// into one edge range and strides over it (every lane takes part in every
// shuffle); `list` is this warp's 3 x 32 words of shared memory.
template <int RP>
__device__ __forceinline__ void pack_warp_push(const PackSeg& g, uint32_t par, int node, uint32_t en, uint32_t lv,
                                               uint32_t* __restrict__ list)
{
    const int lane = threadIdx.x & 31;
    const bool has = (en | lv) != 0u;
    const uint32_t bal = __ballot_sync(kFullP, has);
    if (!bal)
        return;
    const int nev = __popc(bal);
    const int slot = __popc(bal & ((1u << lane) - 1u));
    if (has) {
        list[slot] = (uint32_t)node;
        list[32 + slot] = en;
        list[64 + slot] = lv;
    }
    __syncwarp();
    int64_t lo = 0, len = 0;
    uint32_t me = 0u, ml = 0u;
    if (lane < nev) {
        const int v = (int)list[lane];
        me = list[32 + lane];
        ml = list[64 + lane];
        lo = __ldg(g.out_ptr + v);
        len = __ldg(g.out_ptr + v + 1) - lo;
    }
    int64_t off = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFullP, off, o);
        if (lane >= o)
            off += y;
    }
    const int64_t tot = __shfl_sync(kFullP, off, 31);
    off -= len;
    for (int64_t q0 = 0; q0 < tot; q0 += 32) {
        const int64_t q = q0 + lane;
        int l = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int64_t o = __shfl_sync(kFullP, off, l + st);
            if (o <= q)
                l += st;
        }
        const int64_t lo_l = __shfl_sync(kFullP, lo, l);
        const int64_t off_l = __shfl_sync(kFullP, off, l);
        const uint32_t en_l = __shfl_sync(kFullP, me, l);
        const uint32_t lv_l = __shfl_sync(kFullP, ml, l);
        if (q < tot)
            pack_push_edge<RP>(g, par, (uint32_t)__ldg(g.out_col + lo_l + (q - off_l)), en_l, lv_l);
    }
    __syncwarp();     // the list is reused by the warp's next item
}

// bytes of v equal to b -> 0xff (per byte, b < 256)
__device__ __forceinline__ uint64_t eq_bytes(uint64_t v, uint32_t b)
{
    const uint32_t bb = b * 0x01010101u;
    return (uint64_t)__vcmpeq4((uint32_t)v, bb) | ((uint64_t)__vcmpeq4((uint32_t)(v >> 32), bb) << 32);
}

// bit q of the result = top bit of byte q (bytes 0x00 or 0xff)
__device__ __forceinline__ uint32_t bytes_to_bits(uint64_t m)
{
    const uint32_t lo = (((uint32_t)m & 0x01010101u) * 0x01020408u) >> 24;
    const uint32_t hi = (((uint32_t)(m >> 32) & 0x01010101u) * 0x01020408u) >> 24;
    return lo | (hi << 4);
}

// What a packed warp keeps in shared memory while it processes one group of
// 8 replicates of its 32 nodes: per node slot (lane * 8 + q) the state, the
// count, the age and the decision; the queue of draw units; the replicates'
// scenario headers (probability tables, Philox key, replicate, step size)
// and the lanes' original node ids.
struct PackWarp {
    uint8_t xb[256];
    uint8_t cb[256];
    uint8_t fb[256];
    float age[256];
    uint16_t q[256];           // draw unit: lane | quad << 5 | replicate mask << 6
    uint32_t orig[32];
    // scenario headers of the segment the warp works on (cached across its
    // items): the first 48 bytes of the PackScen of replicate r, and bit j of
    // share = replicates 4j .. 4j+3 share key and Philox counter word
    uint4 sc[kPackMaxR][3];
    const PackScen* sc_src;
    uint32_t share;
    // adaptive segments: this step's size per replicate, and the warp's
    // running maximum of each replicate's rates, added into lam_out (the
    // segment's slot for this step) when the warp moves on
    float dtk[kPackMaxR];
    uint32_t lmx[kPackMaxR];
    uint32_t* lam_out;
};

// the warp's running maxima into the segment's slot (every lane calls this)
__device__ __forceinline__ void pack_flush_lmax(PackWarp& w)
{
    __syncwarp();
    const int lane = threadIdx.x & 31;
    if (w.lam_out && w.lmx[lane])
        atomicMax(w.lam_out + lane, w.lmx[lane]);
    __syncwarp();
}

// the warp's scenario-header cache holds segment g's (loaded when the warp
// moves to another segment; every lane calls this)
template <bool ADAPTIVE>
__device__ __forceinline__ void pack_headers(const PackSeg& g, int64_t k, PackWarp& w)
{
    if (w.sc_src == g.scen)
        return;
    if constexpr (ADAPTIVE)
        pack_flush_lmax(w);
    const int lane = threadIdx.x & 31;
    uint4 h1 = make_uint4(0u, 0u, 0u, 0u);
    if (lane < g.R_pad) {
        const uint4* src = reinterpret_cast<const uint4*>(g.scen + lane);
        w.sc[lane][0] = __ldg(src);
        h1 = __ldg(src + 1);
        w.sc[lane][1] = h1;
        const uint4 h2 = __ldg(src + 2);
        w.sc[lane][2] = h2;
        if constexpr (ADAPTIVE)
            w.dtk[lane] = pack_dt_of(__ldg(g.lam + ((k + 2) % 3) * g.R_pad + lane), __uint_as_float(h2.z),
                                     __uint_as_float(h2.w), __uint_as_float(h1.w));
    }
    if constexpr (ADAPTIVE) {
        w.lmx[lane] = 0u;
        if (lane == 0)
            w.lam_out = g.lam + (k % 3) * g.R_pad;
    }
    const int lead = lane & ~3;
    const uint32_t k0 = __shfl_sync(kFullP, h1.x, lead), k1 = __shfl_sync(kFullP, h1.y, lead);
    const uint32_t c2 = __shfl_sync(kFullP, h1.z >> 2, lead);
    const uint32_t same = __ballot_sync(kFullP, lane < g.R_pad && h1.x == k0 && h1.y == k1 && (h1.z >> 2) == c2);
    uint32_t share = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        share |= ((same >> (4 * j)) & 0xfu) == 0xfu ? (1u << j) : 0u;
    if (lane == 0) {
        w.share = share;
        w.sc_src = g.scen;
    }
    __syncwarp();
}

// Bernoulli probability of replicate q of a slot from its scenario header
// (tables; a miss -- an age off the tabulated sequence -- evaluates the law)
__device__ __forceinline__ float pack_p_hdr(const PackWarp& w, const PackScen& S, int r, int x, float age,
                                            uint32_t c)
{
    if (x == kS) {
        const float* ps = reinterpret_cast<const float*>(((uint64_t)w.sc[r][0].w << 32) | w.sc[r][0].z);
        return __ldg(ps + c);                    // c in 1..255 (thread-class in-degrees are <= 255)
    }
    const float4* pt = reinterpret_cast<const float4*>(((uint64_t)w.sc[r][0].y << 32) | w.sc[r][0].x);
    const float inv_dt = __uint_as_float(w.sc[r][2].y);
    const int n = __float2int_rn(__fmul_rn(age, inv_dt));
    if ((unsigned)n < (unsigned)kPTableN) {
        const float2 e = __ldg(reinterpret_cast<const float2*>(pt + (x == kI ? kPTableN : 0) + n));
        if (e.x == age)
            return e.y;
    }
    return pack_p(S, x, age, 0u);              // slot 1, else direct evaluation (rare)
}

// One group of 8 replicates (b) of the warp's 32 nodes: classification of
// the group's states and counts eight replicates at a time, a queue of draw
// units shared by the warp's lanes (one Philox call serves the replicates of
// a quad that share key and counter), then transitions, ages and the
// per-replicate transition counts. Every lane calls this.
template <typename AgeT, bool ADAPTIVE, bool SHED>
__device__ __forceinline__ void pack_group(const PackSeg& g, int64_t k, int b, bool valid, uint64_t xv, uint64_t cb,
                                           AgeT* __restrict__ Ag, uint8_t* __restrict__ Xg, PackWarp& w,
                                           uint32_t& newmask, uint32_t& oldmask, const AgeVec8<AgeT>* pre,
                                           const float* __restrict__ rsw, AgeT* __restrict__ Rg)
{
    const int lane = threadIdx.x & 31;
    const int slot0 = lane * 8;
    __syncwarp();                  // the previous group has finished with w
    const uint64_t sM = eq_bytes(xv, kS), eM = eq_bytes(xv, kE), iM = eq_bytes(xv, kI);
    const uint64_t eiM = eM | iM;
    uint32_t need;
    if constexpr (SHED) {
        // S replicates under pressure: a positive FP32 sum of infectivities
        // (rsw[r * 32 + lane] = replicate r's sum, this lane's node)
        const uint32_t sb = bytes_to_bits(sM);
        uint32_t sp = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (((sb >> q) & 1u) && rsw[(b * 8 + q) * 32 + lane] > 0.0f)
                sp |= 1u << q;
        need = bytes_to_bits(eiM) | sp;
    } else {
        need = bytes_to_bits(eiM) | bytes_to_bits(sM & ~eq_bytes(cb, 0u));
    }
    if (!valid)
        need = 0u;
    // quads of the group's replicates that share key and Philox counter
    // word (rep >> 2) draw once
    const uint32_t share = (w.share >> (2 * b)) & 3u;
    const bool anyEI = valid && eiM != 0ull;
    if (anyEI) {
        AgeVec8<AgeT> ag;
        if (pre)
            ag = *pre;
        else
            ag.load(Ag);
        *reinterpret_cast<float4*>(w.age + slot0) = make_float4(ag.v[0], ag.v[1], ag.v[2], ag.v[3]);
        *reinterpret_cast<float4*>(w.age + slot0 + 4) = make_float4(ag.v[4], ag.v[5], ag.v[6], ag.v[7]);
    }
    *reinterpret_cast<uint64_t*>(w.xb + slot0) = xv;
    *reinterpret_cast<uint64_t*>(w.cb + slot0) = cb;
    *reinterpret_cast<uint64_t*>(w.fb + slot0) = 0ull;
    // draw units of this lane: a shared quad's needing replicates together,
    // else one unit per needing replicate
    const uint32_t m0 = need & 0xfu, m1 = need >> 4;
    const int nu = (m0 ? ((share & 1u) ? 1 : __popc(m0)) : 0) + (m1 ? ((share & 2u) ? 1 : __popc(m1)) : 0);
    uint32_t incl = (uint32_t)nu;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullP, incl, o);
        if (lane >= o)
            incl += y;
    }
    const int total = (int)__shfl_sync(kFullP, incl, 31);
    {
        int at = (int)incl - nu;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            uint32_t m = j ? m1 : m0;
            if (!m)
                continue;
            if ((share >> j) & 1u) {
                w.q[at++] = (uint16_t)((uint32_t)lane | ((uint32_t)j << 5) | (m << 6));
            } else {
                while (m) {
                    const uint32_t bit = m & (0u - m);
                    m ^= bit;
                    w.q[at++] = (uint16_t)((uint32_t)lane | ((uint32_t)j << 5) | (bit << 6));
                }
            }
        }
    }
    __syncwarp();
    for (int e = lane; e < total; e += 32) {
        const uint32_t unit = w.q[e];
        const int L = (int)(unit & 31u), quad = (int)((unit >> 5) & 1u);
        uint32_t m = unit >> 6;
        const int q0 = quad * 4 + __ffs(m) - 1;
        const uint4 h1 = w.sc[b * 8 + q0][1];
        const uint4 ph = philox4x32_10(make_uint4(w.orig[L], (uint32_t)k, h1.z >> 2, 0u), h1.x, h1.y);
        while (m) {
            const int i = __ffs(m) - 1;
            m &= m - 1u;
            const int q = quad * 4 + i, s_ = L * 8 + q;
            float p;
            if constexpr (ADAPTIVE) {
                const int x = w.xb[s_];
                float lam;
                if (x == kS)
                    lam = SHED ? rsw[(b * 8 + q) * 32 + L]
                               : __fmul_rn(__uint_as_float(w.sc[b * 8 + q][2].x), (float)w.cb[s_]);
                else
                    lam = pack_rate_ei(g.scen[b * 8 + q].M, x, w.age[s_]);
                if (lam > 0.0f)
                    atomicMax(&w.lmx[b * 8 + q], __float_as_uint(lam));
                p = p_of_rate_dt(lam, w.dtk[b * 8 + q]);
            } else if (SHED && w.xb[s_] == kS) {
                p = p_of_rate_dt(rsw[(b * 8 + q) * 32 + L], __uint_as_float(w.sc[b * 8 + q][1].w));
            } else {
                p = pack_p_hdr(w, g.scen[b * 8 + q], b * 8 + q, w.xb[s_], w.age[s_], (uint32_t)w.cb[s_]);
            }
            const uint32_t sel = w.sc[b * 8 + q][1].z & 3u;
            const uint32_t word = sel == 0 ? ph.x : sel == 1 ? ph.y : sel == 2 ? ph.z : ph.w;
            w.fb[s_] = (float)(word >> 8) * 5.9604644775390625e-08f < p ? 0xffu : 0u;
        }
    }
    __syncwarp();
    // transitions: every firing replicate moves on (SEIR: +1; SIR: S -> I is
    // +2, I -> R +1); ages restart at 0 on firing, else E/I ages advance by
    // their scenario's step
    const uint64_t F = valid ? *reinterpret_cast<const uint64_t*>(w.fb + slot0) : 0ull;
    uint64_t inc = F & 0x0101010101010101ull;
    if (g.model != kSEIR)
        inc += F & sM & 0x0101010101010101ull;
    const uint64_t xn = xv + inc;                       // no byte carries: R never fires
    if (valid && F)
        *reinterpret_cast<uint64_t*>(Xg) = xn;
    if (anyEI) {
        const uint32_t fb = bytes_to_bits(F), eb = bytes_to_bits(eiM);
        AgeVec8<AgeT> ag;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float dtq = ADAPTIVE ? w.dtk[b * 8 + q] : __uint_as_float(w.sc[b * 8 + q][1].w);
            ag.v[q] = ((fb >> q) & 1u) ? 0.0f : (((eb >> q) & 1u) ? __fadd_rn(w.age[slot0 + q], dtq) : 0.0f);
        }
        ag.store(Ag);
    }
    newmask |= bytes_to_bits(eq_bytes(xn, kI)) << (b * 8);
    oldmask |= bytes_to_bits(iM) << (b * 8);
    if constexpr (SHED) {
        // the next step's infectivity of the replicates now in I, from their
        // new ages as stored (the others are never read: their mask bit is 0)
        const uint32_t inb = valid ? bytes_to_bits(eq_bytes(xn, kI)) : 0u;
        if (inb) {
            const uint32_t fb = bytes_to_bits(F);
            AgeVec8<AgeT> rv;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                rv.v[q] = 0.0f;
                if ((inb >> q) & 1u) {
                    const float dtq = ADAPTIVE ? w.dtk[b * 8 + q] : __uint_as_float(w.sc[b * 8 + q][1].w);
                    const float na = ((fb >> q) & 1u) ? 0.0f : __fadd_rn(w.age[slot0 + q], dtq);
                    rv.v[q] = pack_rho_of<AgeT>(g.scen[b * 8 + q], na);
                }
            }
            rv.store(Rg);
        }
    }
    // per-replicate transitions of this group, summed over the warp: the
    // fired masks (0xff bytes) become 0/1 bytes, and one warp sum per word
    // adds four replicates' counts at once (at most 32 per byte, no carry)
    const uint64_t one = 0x0101010101010101ull;
    const uint64_t tS = F & sM & one, tE = F & eM & one, tI = F & iM & one;
    if (!__any_sync(kFullP, (tS | tE | tI) != 0ull))
        return;
    const uint32_t s0 = __reduce_add_sync(kFullP, (uint32_t)tS), s1 = __reduce_add_sync(kFullP, (uint32_t)(tS >> 32));
    const uint32_t s2 = __reduce_add_sync(kFullP, (uint32_t)tE), s3 = __reduce_add_sync(kFullP, (uint32_t)(tE >> 32));
    const uint32_t s4 = __reduce_add_sync(kFullP, (uint32_t)tI), s5 = __reduce_add_sync(kFullP, (uint32_t)(tI >> 32));
    // lane f * 8 + q adds field f (S ->, E -> I, I -> R) of replicate b * 8 + q
    if (lane < 24) {
        const int f = lane >> 3, q = lane & 7;
        const uint32_t word = f == 0 ? (q < 4 ? s0 : s1) : f == 1 ? (q < 4 ? s2 : s3) : (q < 4 ? s4 : s5);
        const uint32_t v = (word >> (8 * (q & 3))) & 0xffu;
        if (v)
            atomicAdd(g.deltas + ((k & 1) * g.R_pad + b * 8 + q) * 3 + f, (unsigned long long)v);
    }
}

// SELL slice: lane = node, each lane carries all RP replicates of its node.
// One column load and one RP-bit mask load per edge serve every replicate;
// the mask bits are spread into byte counters (8 per 64-bit word) through a
// 256-entry table in shared memory. Replicates are then processed in groups
// of 8 with vector loads and stores of their states and ages; one Philox
// call serves the replicates that share a key and a counter (rep / 4).
//
// Push form (PUSH): instead of the row gather, each S replicate's count is
// its stored count plus the +1 tally minus the -1 tally of the previous
// step's pushes (bytewise on 8 replicates at once: every byte stays within
// 0..255, so no borrow or carry crosses bytes); replicates that enter or
// leave I are then pushed by the warp along the transposed rows.
// The loads of a slice that need nothing else: its SELL offsets, the lane's
// original node id and its replicates' states. The kernel issues them one
// item ahead, while the warp processes the previous slice.
template <int RP> struct SliceLoads {
    int64_t off, off_end;
    uint32_t orig;
    uint64_t xs[RP / 8];
};

template <int RP, bool PUSH>
__device__ __forceinline__ void slice_loads(const PackSeg& g, int slice, SliceLoads<RP>& L)
{
    const int i = slice * 32 + (threadIdx.x & 31);
    const bool valid = i < g.n_thr;
    L.off = PUSH ? 0 : __ldg(g.sell_off + slice);
    L.off_end = PUSH ? 0 : __ldg(g.sell_off + slice + 1);
    L.orig = (valid && g.perm) ? (uint32_t)__ldg(g.perm + i) : (uint32_t)i;
    const uint64_t* xp = reinterpret_cast<const uint64_t*>(g.X + (int64_t)i * RP);
#pragma unroll
    for (int b = 0; b < RP / 8; ++b)
        L.xs[b] = valid ? xp[b] : 0x0303030303030303ull;
}

template <typename AgeT, int RP, bool PUSH, bool ADAPTIVE, bool SHED>
__device__ __forceinline__ void pack_slice(const PackSeg& g, int64_t k, int slice, const SliceLoads<RP>& L,
                                           const uint64_t* __restrict__ lut, PackWarp& pw,
                                           uint32_t* __restrict__ wlist, float* __restrict__ rsw)
{
    using MT = typename MaskOf<RP>::T;
    constexpr int NB = RP / 8;
    constexpr int B = 12;
    const int lane = threadIdx.x & 31;
    const int i = slice * 32 + lane;
    const bool valid = i < g.n_thr;
    const MT* __restrict__ mk = static_cast<const MT*>(g.mask[k & 1]);
    MT* __restrict__ mkn = static_cast<MT*>(g.mask[(k + 1) & 1]);
    const int64_t off = L.off, off_end = L.off_end;
    const uint32_t orig = L.orig;
    uint64_t xs[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b)
        xs[b] = L.xs[b];
    bool allR = true, anyS = false;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        allR &= xs[b] == 0x0303030303030303ull;
        anyS |= has_byte(xs[b], (uint32_t)kS);
    }
    if (__all_sync(kFullP, allR)) {
        if (!PUSH && valid)
            mkn[i] = (MT)0;
        return;
    }
    // ages are read and written only for groups holding an E or I
    // replicate: the age slot of S and R replicates is always 0, and a
    // transition from S leaves it at 0
    AgeT* __restrict__ Abase = static_cast<AgeT*>(g.A) + (int64_t)i * RP;
    uint8_t* Xb = g.X + (int64_t)i * RP;
    // the first group's ages are issued before the neighbour gather so that
    // the two overlap
    AgeVec8<AgeT> ag0;
    const bool ei0 = valid && (has_byte(xs[0], (uint32_t)kE) || has_byte(xs[0], (uint32_t)kI));
    if (ei0)
        ag0.load(Abase);
    pack_headers<ADAPTIVE>(g, k, pw);
    uint64_t cnt[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b)
        cnt[b] = 0ull;
    if (PUSH && anyS && valid) {
        const uint32_t par = (uint32_t)(k & 1);
        uint64_t* cp = reinterpret_cast<uint64_t*>(g.pc8 + (int64_t)i * RP);
        uint4* pp = reinterpret_cast<uint4*>(g.ppd[par ^ 1u] + (int64_t)i * RP);
        bool nz = false;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint64_t c8 = cp[b];
            const uint4 w = pp[b];
            const uint64_t plus = (uint64_t)__byte_perm(w.x, w.y, 0x6420u) | ((uint64_t)__byte_perm(w.z, w.w, 0x6420u) << 32);
            const uint64_t minus = (uint64_t)__byte_perm(w.x, w.y, 0x7531u) | ((uint64_t)__byte_perm(w.z, w.w, 0x7531u) << 32);
            const uint64_t m = s_bytes(xs[b]);
            cnt[b] = ((c8 & m) - (minus & m)) + (plus & m);
            nz |= (w.x | w.y | w.z | w.w) != 0u;
        }
        if (nz) {
            // fold the tallies into the counts and clear them for the next step
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                cp[b] = cnt[b];
                pp[b] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
    if constexpr (PUSH) {
        // nothing can happen in a slice with no E or I replicate whose S
        // replicates all have count 0 (their tallies are folded above): no
        // draw, no transition, no write, no push
        bool busy = false;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            busy |= cnt[b] != 0ull || has_byte(xs[b], (uint32_t)kE) || has_byte(xs[b], (uint32_t)kI);
        if (!__any_sync(kFullP, busy))
            return;
    }
    if (SHED && anyS) {
        // Eq. 3 with the infectivities of Eq. 8: each S replicate r sums, in
        // FP32 and in row order, the stored rho of the in-neighbours whose
        // replicate r is infectious (the single-realisation step's order)
#pragma unroll
        for (int r = 0; r < RP; ++r)
            rsw[r * 32 + lane] = 0.0f;
        uint32_t sbits = 0u;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            sbits |= bytes_to_bits(s_bytes(xs[b])) << (8 * b);
        const AgeT* __restrict__ rho = static_cast<const AgeT*>(g.rho[k & 1]);
        const int w = (int)((off_end - off) >> 5);
        const int32_t* __restrict__ p = g.sell_col + off + lane;
        for (int t0 = 0; t0 < w; t0 += B) {
            int32_t jj[B];
#pragma unroll
            for (int u = 0; u < B; ++u)
                jj[u] = (t0 + u < w) ? __ldg(p + 32 * (t0 + u)) : g.sentinel;
#pragma unroll
            for (int u = 0; u < B; ++u) {
                uint32_t hit = (uint32_t)__ldg(mk + jj[u]) & sbits;   // the sentinel's mask is always 0
                while (hit) {
                    const int r = __ffs(hit) - 1;
                    hit &= hit - 1u;
                    rsw[r * 32 + lane] = __fadd_rn(rsw[r * 32 + lane],
                                                   AgeIO<AgeT>::load(rho[(int64_t)jj[u] * RP + r]));
                }
            }
        }
    } else if (!PUSH && anyS) {
        const int w = (int)((off_end - off) >> 5);
        const int32_t* __restrict__ p = g.sell_col + off + lane;
        for (int t0 = 0; t0 < w; t0 += B) {
            int32_t jj[B];
#pragma unroll
            for (int u = 0; u < B; ++u)
                jj[u] = (t0 + u < w) ? __ldg(p + 32 * (t0 + u)) : g.sentinel;
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const uint32_t m = (uint32_t)__ldg(mk + jj[u]);   // the sentinel's mask is always 0
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    cnt[b] += lut[(m >> (8 * b)) & 0xffu];
            }
        }
    }
    uint32_t newmask = 0, oldmask = 0;
    __syncwarp();                  // the warp's previous item has finished with pw
    pw.orig[lane] = orig;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (b * 8 >= g.R)
            break;
        pack_group<AgeT, ADAPTIVE, SHED>(g, k, b, valid, xs[b], cnt[b], Abase + b * 8, Xb + b * 8, pw, newmask,
                                         oldmask, b == 0 && ei0 ? &ag0 : nullptr, rsw,
                                         SHED ? static_cast<AgeT*>(g.rho[(k + 1) & 1]) + (int64_t)i * RP + b * 8
                                              : nullptr);
    }
    if constexpr (PUSH) {
        const uint32_t en = valid ? newmask & ~oldmask : 0u, lv = valid ? oldmask & ~newmask : 0u;
        pack_warp_push<RP>(g, (uint32_t)(k & 1), i, en, lv, wlist);
    } else {
        if (valid)
            mkn[i] = (MT)newmask;
    }
}

// hub row: one warp, lane r < L is replicate r; 32 edges per window
template <typename AgeT, int L, bool ADAPTIVE>
__device__ __forceinline__ void pack_hub_row(const PackSeg& g, int64_t k, int row)
{
    using MT = typename MaskOf<L>::T;
    constexpr int U = 4;                             // windows in flight
    const int lane = threadIdx.x & 31;
    const int i = g.n_thr + row;
    const bool mine = lane < L;
    const int64_t off_state = (int64_t)i * L + lane;
    AgeT* __restrict__ A = static_cast<AgeT*>(g.A);
    const MT* __restrict__ mk = static_cast<const MT*>(g.mask[k & 1]);
    MT* __restrict__ mkn = static_cast<MT*>(g.mask[(k + 1) & 1]);
    const int x = mine ? (int)g.X[off_state] : kR;
    float age = 0.0f;
    if (x == kE || x == kI)
        age = AgeIO<AgeT>::load(A[off_state]);
    const uint32_t sm = __ballot_sync(kFullP, x == kS);
    uint32_t c = 0;
    if (sm) {
        const int64_t e0 = __ldg(g.m_ptr + row), e1 = __ldg(g.m_ptr + row + 1);
        for (int64_t w0 = e0; w0 < e1; w0 += 32 * U) {
            uint32_t m[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = w0 + 32 * u + lane;
                const int32_t col = e < e1 ? __ldg(g.m_col + e) : g.sentinel;
                m[u] = (uint32_t)__ldg(mk + col);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t todo = sm;
                while (todo) {                        // one ballot per S replicate
                    const int rr = __ffs(todo) - 1;
                    todo &= todo - 1u;
                    const uint32_t bal = __ballot_sync(kFullP, (m[u] >> rr) & 1u);
                    if (lane == rr)
                        c += __popc(bal);
                }
            }
        }
    }
    const PackScen& S = g.scen[mine ? lane : 0];
    PackTail t{x, 0.0f, false};
    if (mine)
        t = ADAPTIVE ? pack_tail_adaptive(g, k, lane, x, age, c, i) : pack_tail(S, g.model, x, age, c, g.perm, i, (uint32_t)k);
    if (mine) {
        if (t.x != x)
            g.X[off_state] = (uint8_t)t.x;
        if (t.fired || x == kE || x == kI)
            A[off_state] = AgeIO<AgeT>::store(t.age);
    }
    const uint32_t b = __ballot_sync(kFullP, mine && t.x == kI);
    if (lane == 0)
        mkn[i] = (MT)b;
    if (mine)
        add_deltas(g, k, lane, t.fired && x == kS, t.fired && x == kE, t.fired && x == kI);
}

// hub row with a shedding profile: lane r < L is replicate r. Each S
// replicate's pressure is the FP32 sum of the stored rho of its infectious
// in-neighbours, summed in the order of the single-realisation merge kernel,
// so that a packed replicate keeps the bits it has alone: the row's edges go
// in 32-edge windows aligned to the merge CSR (a segmented scan of fixed tree
// shape inside each window), windows fold in order within each
// kMergeEdgesPerWarp-edge warp range, warp ranges within each kMergeEPB-edge
// chunk, and chunks in order.
template <typename AgeT, int L, bool ADAPTIVE>
__device__ __forceinline__ void pack_hub_row_shed(const PackSeg& g, int64_t k, int row)
{
    using MT = typename MaskOf<L>::T;
    const int lane = threadIdx.x & 31;
    const int i = g.n_thr + row;
    const bool mine = lane < L;
    const int64_t off_state = (int64_t)i * L + lane;
    AgeT* __restrict__ A = static_cast<AgeT*>(g.A);
    const MT* __restrict__ mk = static_cast<const MT*>(g.mask[k & 1]);
    MT* __restrict__ mkn = static_cast<MT*>(g.mask[(k + 1) & 1]);
    const AgeT* __restrict__ rho = static_cast<const AgeT*>(g.rho[k & 1]);
    const int x = mine ? (int)g.X[off_state] : kR;
    float age = 0.0f;
    if (x == kE || x == kI)
        age = AgeIO<AgeT>::load(A[off_state]);
    const uint32_t sm = __ballot_sync(kFullP, x == kS);
    float lam = 0.0f;                       // lane r: replicate r's pressure
    if (sm) {
        const int64_t e0 = __ldg(g.m_ptr + row), e1 = __ldg(g.m_ptr + row + 1);
        float accW = 0.0f, accC = 0.0f;
        int64_t curW = -1, curC = -1;
        bool started = false;
        for (int64_t wb = e0 & ~(int64_t)31; wb < e1; wb += 32) {
            const int64_t ws = wb / kMergeEdgesPerWarp, wc = wb / kMergeEPB;
            if (ws != curW) {
                if (curW >= 0)
                    accC = __fadd_rn(accC, accW);
                accW = 0.0f;
                curW = ws;
                if (wc != curC) {
                    if (curC >= 0) {
                        lam = started ? __fadd_rn(lam, accC) : accC;
                        started = true;
                    }
                    accC = 0.0f;
                    curC = wc;
                }
            }
            const int l0 = (int)max((int64_t)0, e0 - wb), h0 = (int)min((int64_t)32, e1 - wb);
            const int64_t e = wb + lane;
            const bool in = lane >= l0 && lane < h0;
            const int32_t col = in ? __ldg(g.m_col + e) : g.sentinel;
            const uint32_t m = (uint32_t)__ldg(mk + col);      // the sentinel's mask is always 0
            uint32_t todo = sm;
            while (todo) {
                const int rr = __ffs(todo) - 1;
                todo &= todo - 1u;
                float v = ((m >> rr) & 1u) ? AgeIO<AgeT>::load(rho[(int64_t)col * L + rr]) : 0.0f;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const float t = __shfl_up_sync(kFullP, v, d);
                    if (lane - d >= l0)
                        v = __fadd_rn(v, t);
                }
                const float seg = __shfl_sync(kFullP, v, h0 - 1);
                if (lane == rr)
                    accW = __fadd_rn(accW, seg);
            }
        }
        accC = __fadd_rn(accC, accW);
        lam = started ? __fadd_rn(lam, accC) : accC;
    }
    const PackScen& S = g.scen[mine ? lane : 0];
    PackTail t{x, 0.0f, false};
    if (mine) {
        if constexpr (ADAPTIVE) {
            t = pack_tail_adaptive_rate(g, k, lane, x, age, x == kS ? lam : 0.0f, i);
        } else {
            const float p = x == kS ? p_of_rate(S.M, lam) : pack_p(S, x, age, 0u);
            t = pack_tail_p(S, g.model, x, age, p, g.perm, i, (uint32_t)k);
        }
    }
    if (mine) {
        if (t.x != x)
            g.X[off_state] = (uint8_t)t.x;
        if (t.fired || x == kE || x == kI)
            A[off_state] = AgeIO<AgeT>::store(t.age);
        if (t.x == kI)
            static_cast<AgeT*>(g.rho[(k + 1) & 1])[off_state] = AgeIO<AgeT>::store(pack_rho_of<AgeT>(S, t.age));
    }
    const uint32_t b = __ballot_sync(kFullP, mine && t.x == kI);
    if (lane == 0)
        mkn[i] = (MT)b;
    if (mine)
        add_deltas(g, k, lane, t.fired && x == kS, t.fired && x == kE, t.fired && x == kI);
}

// hub row, push form: lane r < L is replicate r; its count is folded from its
// pending tallies, and the replicates that enter or leave I are pushed by the
// whole warp along the node's transposed row
template <typename AgeT, int L, bool ADAPTIVE>
__device__ __forceinline__ void pack_hub_row_push(const PackSeg& g, int64_t k, int row)
{
    const int lane = threadIdx.x & 31;
    const int i = g.n_thr + row;
    const bool mine = lane < L;
    const uint32_t par = (uint32_t)(k & 1);
    const int64_t off_state = (int64_t)i * L + lane;
    AgeT* __restrict__ A = static_cast<AgeT*>(g.A);
    const int x = mine ? (int)g.X[off_state] : kR;
    float age = 0.0f;
    if (x == kE || x == kI)
        age = AgeIO<AgeT>::load(A[off_state]);
    uint32_t c = 0u;
    if (x == kS) {
        const int64_t h = (int64_t)row * L + lane;
        unsigned long long* pr = g.phpd[par ^ 1u] + h;
        const unsigned long long d = *pr;
        c = g.phc[h];
        if (d) {
            c = c + (uint32_t)(d & 0xffffffffull) - (uint32_t)(d >> 32);
            g.phc[h] = c;
            *pr = 0ull;
        }
    }
    const PackScen& S = g.scen[mine ? lane : 0];
    PackTail t{x, 0.0f, false};
    if (mine)
        t = ADAPTIVE ? pack_tail_adaptive(g, k, lane, x, age, c, i) : pack_tail(S, g.model, x, age, c, g.perm, i, (uint32_t)k);
    if (mine) {
        if (t.x != x)
            g.X[off_state] = (uint8_t)t.x;
        if (t.fired || x == kE || x == kI)
            A[off_state] = AgeIO<AgeT>::store(t.age);
        add_deltas(g, k, lane, t.fired && x == kS, t.fired && x == kE, t.fired && x == kI);
    }
    const uint32_t en = __ballot_sync(kFullP, mine && t.x == kI && x != kI);
    const uint32_t lv = __ballot_sync(kFullP, mine && x == kI && t.x != kI);
    if (en | lv) {
        const int64_t e0 = __ldg(g.out_ptr + i), e1 = __ldg(g.out_ptr + i + 1);
        for (int64_t e = e0 + lane; e < e1; e += 32)
            pack_push_edge<L>(g, par, (uint32_t)__ldg(g.out_col + e), en, lv);
    }
}

// integrate the deltas of the segment's previous step and write its row
__device__ __forceinline__ void pack_integrate(const PackSeg& g, int64_t k)
{
    const int lane = threadIdx.x & 31;
    if (k <= g.kmin || k > g.kend || lane >= g.R_pad)
        return;
    unsigned long long* d = g.deltas + (((k - 1) & 1) * g.R_pad + lane) * 3;
    const uint32_t l = (uint32_t)d[0], ei = (uint32_t)d[1], ir = (uint32_t)d[2];
    d[0] = 0ull;
    d[1] = 0ull;
    d[2] = 0ull;
    uint32_t* cnt = g.counts + lane * 4;
    uint32_t c0 = cnt[0], c1 = cnt[1], c2 = cnt[2], c3 = cnt[3];
    c0 -= l;
    if (g.model == kSEIR) {
        c1 += l - ei;
        c2 += ei - ir;
    } else {
        c2 += l - ir;
    }
    c3 += ir;
    cnt[0] = c0; cnt[1] = c1; cnt[2] = c2; cnt[3] = c3;
    if (g.out) {
        uint32_t* o = g.out + ((k - g.kmin) * g.R_pad + lane) * 4;
        o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
    }
    if (g.lam) {
        // the previous step's size (from the rates of the step before it)
        // into the replicate's clock; that slot then takes step k + 1's rates
        uint32_t* slot = g.lam + ((k + 1) % 3) * g.R_pad + lane;
        const PackScen& S = g.scen[lane];
        g.time[lane] += (double)pack_dt_of(*slot, S.eps, S.delta, S.M.dt);
        *slot = 0u;
    }
}

}  // namespace

// Minimum resident blocks per SM of the packed step, by replicate width: the
// register budget that measured fastest for each (80 and 96 registers).
#ifndef FS_PACK_MIN_BLOCKS8
#define FS_PACK_MIN_BLOCKS8 6
#endif
template <int RP> struct PackOcc { static constexpr int kMinBlocks = RP == 8 ? FS_PACK_MIN_BLOCKS8 : 5; };

template <typename AgeT, int RP, int FORM, bool ADAPTIVE>
__global__ void __launch_bounds__(kPackThreads, PackOcc<RP>::kMinBlocks) pack_step_kernel(const __grid_constant__ PackArgs a)
{
    // pressure form: 0 gather, 1 push, 2 gather with a shedding profile
    constexpr bool PUSH = FORM == 1, SHED = FORM == 2;
    // per warp, with a shedding profile: the FP32 pressure of every (replicate,
    // node) of its slice, [RP][32]
    __shared__ float s_rs[SHED ? (kPackThreads / 32) * RP * 32 : 1];
    // byte r of lut[m] is bit r of m: spreads an 8-replicate mask into byte counters
    __shared__ uint64_t lut[256];
    // per warp: one 8-replicate group of its slice (states, counts, ages,
    // decisions, the draw queue, the replicates' scenario headers)
    __shared__ PackWarp s_pw[kPackThreads / 32];
    // per warp: the push events of one slice (node, entering mask, leaving mask)
    __shared__ uint32_t s_ev[kPackThreads / 32][3 * 32];
    PackWarp& pw = s_pw[threadIdx.x >> 5];
    if ((threadIdx.x & 31) == 0) {
        pw.sc_src = nullptr;
        pw.lam_out = nullptr;
    }
    uint32_t* wlist = s_ev[threadIdx.x >> 5];
    float* rsw = SHED ? s_rs + (threadIdx.x >> 5) * RP * 32 : nullptr;
    for (int m = threadIdx.x; m < 256; m += blockDim.x) {
        uint64_t v = 0;
        for (int r = 0; r < 8; ++r)
            v |= (uint64_t)((m >> r) & 1) << (8 * r);
        lut[m] = v;
    }
    __syncthreads();
    constexpr int c = ((RP == 8 ? 0 : RP == 16 ? 1 : 2) * 3 + FORM) * 2 + (ADAPTIVE ? 1 : 0);
    const int64_t G = a.ctl->step + a.j;
    const int s0 = a.cls[c], s1 = a.cls[c + 1];
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // counts of the previous step, one warp per segment
    for (int64_t s = s0 + gw; s < s1; s += W) {
        const PackSeg& g = a.seg[s];
        pack_integrate(g, G - g.join);
    }
    // hub rows (long rows start first), then SELL items
    const int64_t hub0 = __ldg(a.hub_pre + s0), n_hub = __ldg(a.hub_pre + s1);
    const int64_t thr0 = __ldg(a.thr_pre + s0), n_thr = __ldg(a.thr_pre + s1);
    int s = s0;
    for (int64_t it = hub0 + gw; it < n_hub; it += W) {
        while (__ldg(a.hub_pre + s + 1) <= it)
            ++s;
        const PackSeg& g = a.seg[s];
        const int64_t k = G - g.join;
        if (k < g.kmin || k >= g.kend)
            continue;
        if constexpr (PUSH)
            pack_hub_row_push<AgeT, RP, ADAPTIVE>(g, k, (int)(it - __ldg(a.hub_pre + s)));
        else if constexpr (SHED)
            pack_hub_row_shed<AgeT, RP, ADAPTIVE>(g, k, (int)(it - __ldg(a.hub_pre + s)));
        else
            pack_hub_row<AgeT, RP, ADAPTIVE>(g, k, (int)(it - __ldg(a.hub_pre + s)));
    }
    // one item per 32-node slice; the next item's independent loads are
    // issued before the current one is processed
    s = s0;
    int64_t it = thr0 + gw;
    SliceLoads<RP> cur;
    if (it < n_thr) {
        while (__ldg(a.thr_pre + s + 1) <= it)
            ++s;
        slice_loads<RP, PUSH>(a.seg[s], (int)(it - __ldg(a.thr_pre + s)), cur);
    }
    while (it < n_thr) {
        const int sc = s;
        const int64_t ic = it;
        it += W;
        SliceLoads<RP> nxt;
        if (it < n_thr) {
            while (__ldg(a.thr_pre + s + 1) <= it)
                ++s;
            slice_loads<RP, PUSH>(a.seg[s], (int)(it - __ldg(a.thr_pre + s)), nxt);
        }
        const PackSeg& g = a.seg[sc];
        const int64_t k = G - g.join;
        if (k >= g.kmin && k < g.kend)
            pack_slice<AgeT, RP, PUSH, ADAPTIVE, SHED>(g, k, (int)(ic - __ldg(a.thr_pre + sc)), cur, lut, pw, wlist,
                                                       rsw);
        cur = nxt;
    }
    if constexpr (ADAPTIVE)
        pack_flush_lmax(pw);
}

// initial packed state of a segment: replicates r < R start in S with the
// index nodes in `index_state`; padding replicates are absorbed (R)
__global__ void pack_init_kernel(uint8_t* X, int n, int R_pad, int R)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < (int64_t)n * R_pad)
        X[t] = (uint8_t)((t % R_pad) < R ? kS : kR);
}

__global__ void pack_index_kernel(uint8_t* X, const int32_t* idx, int64_t n_idx, const int32_t* inv, int R_pad, int R,
                                  int state, uint32_t* mask32, uint16_t* mask16, uint8_t* mask8)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_idx)
        return;
    const int o = idx[q];
    const int i = inv ? inv[o] : o;
    for (int r = 0; r < R; ++r)
        X[(int64_t)i * R_pad + r] = (uint8_t)state;
    if (state == kI) {
        const uint32_t bits = R == 32 ? 0xffffffffu : ((1u << R) - 1u);
        if (mask32) mask32[i] = bits;
        if (mask16) mask16[i] = (uint16_t)bits;
        if (mask8) mask8[i] = (uint8_t)bits;
    }
}

// initial counts of a push-form segment (counts zeroed before): every node
// pushes +1, for each replicate in which it is I, into the counts of its
// out-neighbours (bytes of 32-bit words for the thread class: counts never
// exceed the in-degree, so no carry crosses bytes)
__global__ void pack_push_init_kernel(PackSeg g)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n)
        return;
    const int RP = g.R_pad;
    uint32_t im = 0u;
    for (int r = 0; r < RP; ++r)
        im |= (uint32_t)(g.X[i * RP + r] == kI) << r;
    if (!im)
        return;
    const int64_t e0 = g.out_ptr[i], e1 = g.out_ptr[i + 1];
    for (int64_t e = e0; e < e1; ++e) {
        const uint32_t j = (uint32_t)g.out_col[e];
        if (j < (uint32_t)g.n_thr) {
            unsigned int* w = reinterpret_cast<unsigned int*>(g.pc8 + (int64_t)j * RP);
            for (int q = 0; q < RP / 4; ++q) {
                const uint32_t b = (im >> (4 * q)) & 0xfu;
                if (b)
                    atomicAdd(w + q, (b & 1u) | (((b >> 1) & 1u) << 8) | (((b >> 2) & 1u) << 16) |
                                         (((b >> 3) & 1u) << 24));
            }
        } else if (j < (uint32_t)g.n) {
            uint32_t m = im;
            while (m) {
                const int r = __ffs(m) - 1;
                m &= m - 1u;
                atomicAdd(g.phc + (int64_t)(j - (uint32_t)g.n_thr) * RP + r, 1u);
            }
        }
    }
}

cudaError_t launch_pack_push_init(const PackSeg& g, cudaStream_t s)
{
    pack_push_init_kernel<<<(unsigned)((g.n + 255) / 256), 256, 0, s>>>(g);
    g_launch_count += 1;
    return cudaGetLastError();
}

__global__ void pack_advance_kernel(DevCtl* ctl, int K)
{
    if (threadIdx.x == 0)
        ctl->step += K;
}

cudaError_t launch_pack_advance(DevCtl* ctl, int K, cudaStream_t s)
{
    pack_advance_kernel<<<1, 32, 0, s>>>(ctl, K);
    g_launch_count += 1;
    return cudaGetLastError();
}

template <typename AgeT, int FORM, bool ADAPTIVE>
static cudaError_t launch_pack_t(const PackArgs& a, int cls, int grid, cudaStream_t s)
{
    switch (cls) {
    case 0: pack_step_kernel<AgeT, 8, FORM, ADAPTIVE><<<grid, kPackThreads, 0, s>>>(a); break;
    case 1: pack_step_kernel<AgeT, 16, FORM, ADAPTIVE><<<grid, kPackThreads, 0, s>>>(a); break;
    default: pack_step_kernel<AgeT, 32, FORM, ADAPTIVE><<<grid, kPackThreads, 0, s>>>(a); break;
    }
    g_launch_count += 1;
    return cudaGetLastError();
}

template <typename AgeT, int FORM>
static cudaError_t launch_pack_f(const PackArgs& a, int cls, bool adaptive, int grid, cudaStream_t s)
{
    return adaptive ? launch_pack_t<AgeT, FORM, true>(a, cls, grid, s) : launch_pack_t<AgeT, FORM, false>(a, cls, grid, s);
}

template <typename AgeT>
static cudaError_t launch_pack_a(const PackArgs& a, int cls, int form, bool adaptive, int grid, cudaStream_t s)
{
    switch (form) {
    case 1: return launch_pack_f<AgeT, 1>(a, cls, adaptive, grid, s);
    case 2: return launch_pack_f<AgeT, 2>(a, cls, adaptive, grid, s);
    default: return launch_pack_f<AgeT, 0>(a, cls, adaptive, grid, s);
    }
}

cudaError_t launch_pack_step(const PackArgs& a, int cls, int form, bool adaptive, int age_dtype, int grid,
                             cudaStream_t s)
{
    switch (age_dtype) {
    case kAgeF16: return launch_pack_a<__half>(a, cls, form, adaptive, grid, s);
    case kAgeBF16: return launch_pack_a<__nv_bfloat16>(a, cls, form, adaptive, grid, s);
    default: return launch_pack_a<float>(a, cls, form, adaptive, grid, s);
    }
}

// initial infectivity of a segment with a shedding profile: replicates that
// start in I (index nodes with index_state I) get beta s(0) in rho[par]
template <typename AgeT>
__global__ void pack_rho_init_kernel(PackSeg g, uint32_t par)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)g.n * g.R_pad)
        return;
    const int r = (int)(t % g.R_pad);
    if (r < g.R && g.X[t] == kI)
        static_cast<AgeT*>(g.rho[par])[t] = AgeIO<AgeT>::store(pack_rho_of<AgeT>(g.scen[r], 0.0f));
}

cudaError_t launch_pack_rho_init(const PackSeg& g, int age_dtype, uint32_t par, cudaStream_t s)
{
    const int64_t total = (int64_t)g.n * g.R_pad;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    switch (age_dtype) {
    case kAgeF16: pack_rho_init_kernel<__half><<<blocks, 256, 0, s>>>(g, par); break;
    case kAgeBF16: pack_rho_init_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(g, par); break;
    default: pack_rho_init_kernel<float><<<blocks, 256, 0, s>>>(g, par); break;
    }
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_pack_init(uint8_t* X, int n, int R_pad, int R, const int32_t* idx, int64_t n_idx,
                             const int32_t* inv, int state, void* mask, cudaStream_t s)
{
    const int64_t total = (int64_t)n * R_pad;
    pack_init_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, n, R_pad, R);
    g_launch_count += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n_idx == 0)
        return e;
    pack_index_kernel<<<(unsigned)((n_idx + 255) / 256), 256, 0, s>>>(
        X, idx, n_idx, inv, R_pad, R, state, R_pad == 32 ? (uint32_t*)mask : nullptr,
        R_pad == 16 ? (uint16_t*)mask : nullptr, R_pad == 8 ? (uint8_t*)mask : nullptr);
    g_launch_count += 1;
    return cudaGetLastError();
}

int pack_grid(int num_sms, int cls)
{
    int occ = 0;
    cudaError_t e = cls == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pack_step_kernel<float, 8, 0, false>, kPackThreads, 0)
                    : cls == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pack_step_kernel<float, 16, 0, false>, kPackThreads, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pack_step_kernel<float, 32, 0, false>, kPackThreads, 0);
    if (e != cudaSuccess || occ < 1)
        occ = 4;
    return num_sms * occ;
}

}  // namespace fs
