// fs_internal.h -- definitions shared by the CUDA translation units of
// libflashstep (not part of the public C ABI in include/fs.h).
#pragma once

#include <cstdint>

namespace fs {

enum { kS = 0, kE = 1, kI = 2, kR = 3 };
enum { kSIR = 0, kSEIR = 1, kSIS = 2 };
enum { kLawNone = 0, kLawExp = 1, kLawLogNormal = 2, kLawWeibull = 3, kLawErlang = 4 };
enum { kAgeF32 = 0, kAgeF16 = 1, kAgeBF16 = 2 };

// FP32 law constants prepared on the host (double -> float once):
//   EXP:       p0 = rate
//   LOGNORMAL: mu = p0 + p3 and 1/(sigma sqrt 2) = p1 + p4 (hi/lo float
//              pairs), p2 = sqrt(2/pi)/sigma
//   WEIBULL:   p0 = k/s, p1 = 1/s, p2 = k - 1
//   ERLANG:    p0 = rate, k = stages
struct LawF {
    int32_t kind;
    int32_t k;
    float p0, p1, p2, p3, p4;
};

struct ModelF {
    int32_t model;
    float beta;
    float dt;
    float inv_dt;                 // (float)(1/dt): age -> table index
    uint32_t key0, key1, rep;
    LawF lat, inf;
};

constexpr int kWarp = 32;
constexpr int kStepThreads = 256;                 // 8 warps per CTA
constexpr int kStepWarps = kStepThreads / kWarp;
constexpr int kSellSlicesPerCta = kStepWarps;     // one 32-node SELL slice per warp
constexpr int kMergeWindowsPerWarp = 16;          // 16 x 32-edge windows per warp
constexpr int kMergeEdgesPerWarp = kMergeWindowsPerWarp * kWarp;   // 512
constexpr int kMergeEPB = kMergeEdgesPerWarp * kStepWarps;         // 4096 edges per CTA
constexpr int kMinMergeDegree = 32;               // keeps <= 18 rows per warp range
constexpr int kMergeMaxRows = kMergeEPB / kMinMergeDegree + 2;     // rows one chunk can touch
constexpr int kMaxThreadDeg = 255;                // bucket cap of the degree sort
constexpr uint32_t kWaitLimit = 1u << 20;         // bounded mbarrier waits
constexpr int kMaxGraphSteps = 256;              // steps per captured graph / epilogue
constexpr int kPTableN = 4096;                    // age-indexed p entries per law
constexpr int kPSTableN = 256;                    // p of an S node by infectious count
constexpr int kStepCtasPerSm = 5;                 // resident step CTAs per SM (256 thr, <= 48 regs)
constexpr int kSmemThreads = 1024;                // one CTA per SM holding the bitmap in shared memory
constexpr uint32_t kSmemBitmapMaxBytes = 200u * 1024u;   // bitmap sizes staged in shared memory

// Markovian engine: the integer reductions of one state's rates
struct MarkovSums {
    unsigned long long si;        // sum over S nodes of their infectious in-neighbours
    unsigned long long ne, ni;    // |E|, |I|
    unsigned int cmax;            // largest count of an S node
    unsigned int pad_;
};

// Device-resident control block of one simulation (the persistent scalars of
// Algorithm 2: step counter; plus running counts and work accounting).
struct DevCtl {
    int64_t step;                 // index of the next step
    int64_t row;                  // next row of the counts output
    uint32_t* out;                // counts output ((steps+1) x 4) or null
    unsigned long long ds_cur;    // sum of degrees of the current S nodes
    unsigned long long ds_total;  // sum over run steps of ds at step start
    unsigned long long s_total;   // sum over run steps of |S| at step start
    uint32_t counts[4];           // counts of the current state
    int32_t error;                // device error word (0 = ok)
    int32_t pad_;
    // adaptive step: the largest rate of step k goes to lam[k % 3] (FP32
    // bits, atomic max), read by step k + 1 for its size; simulated time
    uint32_t lam[3];
    int32_t pad2_;
    double time;                  // sum of the step sizes since init / set_state
    // active-node compaction: units listed by the refresh of the current
    // launch sequence (moved into act_sum and reset to 0 by the epilogue)
    unsigned long long n_act;
    unsigned long long act_sum;   // sum over launch sequences of n_act
    // Markovian engine: rate sums of step k in mk[k & 1] (step k clears
    // mk[(k + 1) & 1] for the next reduction); events appended by a step
    MarkovSums mk[2];
    unsigned int mk_nev;
    unsigned int pad3_;
    unsigned long long transitions;   // node transitions since init / set_state
    // bounds-checked builds (FS_DEBUG_BOUNDS): the first index a check
    // rejected and the check's site number (kErrBounds in `error`)
    long long dbg_index;
    int32_t dbg_site;
    int32_t pad4_;
};

enum { kErrNone = 0, kErrTmaTimeout = 1, kErrBadState = 2, kErrBadGraph = 3, kErrBounds = 4 };

// sites of the FS_DEBUG_BOUNDS checks (reported with the rejected index)
enum {
    kSiteGroup = 1,        // push step: a group's vector of node slots
    kSiteOutPtr = 2,       // push step: a pushing node's transposed row bounds
    kSiteOutCol = 3,       // push step: a transposed column index
    kSitePushTarget = 4,   // push step: the node a push lands on
    kSiteSellCol = 5,      // gather: a SELL column entry
    kSiteBitmap = 6,       // gather: a bitmap word
};

// Per-step deltas accumulated by the step kernel (atomics, skipped when 0):
// [0] nodes that left S, [1] E -> I, [2] I -> R, [3] sum of degrees of the
// nodes that left S. Each step's row is spread over kDeltaSlots slots
// (uint64 [K][kDeltaSlots][kDeltaFields]): warp w of a step's grid adds its
// totals into slot w mod kDeltaSlots, so that no CTA-wide reduction or
// barrier ends the step and no word takes more than a few dozen atomics; the
// epilogue sums the slots.
constexpr int kDeltaFields = 4;
constexpr int kDeltaSlots = 32;
constexpr int kDeltaRow = kDeltaSlots * kDeltaFields;   // words per step

// Everything the fused step kernel reads, passed by value.
struct StepArgs {
    uint8_t* X;                   // compartments, internal order
    void* A;                      // ages (f32/f16/bf16), internal order
    uint32_t* bm[2];              // infectious bitmaps; step k reads bm[k&1]
    // one-thread-per-node class: SELL-32 over internal ids [0, n_thr)
    const int64_t* sell_off;      // [n_slices + 1] entry offsets
    const int32_t* sell_col;      // column-major 32-wide blocks, padding = sentinel
    int32_t n_thr;
    int32_t n_slices;
    int32_t sentinel;             // id whose bitmap bit is always 0 (= n)
    // merge class: internal ids [m_base, m_base + n_m), CSR rows relative
    int32_t m_base;
    int32_t n_m;
    int32_t n_chunks;             // kMergeEPB-edge chunks
    int32_t n_sell_ctas;
    const int64_t* m_ptr;         // [n_m + 1], m_ptr[0] = 0
    const int32_t* m_col;         // [n_chunks * kMergeEPB], padded with sentinel
    const int32_t* m_warp_row;    // [n_chunks * kStepWarps] row of each warp range start
    const int32_t* m_chunk_last;  // [n_chunks] row containing the chunk's last edge
    int64_t e_m;                  // edges of the merge class
    int32_t* m_cnt;               // [n_m] cross-chunk partial counts (scratch)
    uint32_t* m_tkt;              // [n_m] cross-chunk tickets (scratch)
    const int32_t* perm;          // internal -> original id, null = identity
    const int32_t* deg;           // degree by internal id (work accounting of fired S nodes)
    // Bernoulli probabilities memoised per sim (bit-identical to direct
    // evaluation): ptab[law * kPTableN + n] = (age0, p0, age1, p1), the ages
    // of the fixed-step sequence whose index rint(age / dt) is n (at most two
    // distinct ages share an index: the sequence is monotone and its steps
    // are at least half an index apart; NaN age = empty slot); law 0 =
    // latent, 1 = infectious; ps[c] = p of an S node with c infectious
    // in-neighbours
    const float4* ptab;
    const float* ps;
    int32_t spw;                  // SELL slices per warp
    uint32_t bm_bytes;            // bitmap bytes copied to shared memory (multiple of 16)
    uint32_t smem_min_s;          // stage the bitmap when at least this many nodes are S
    ModelF M;
    DevCtl* ctl;
    unsigned long long* deltas;   // [K][kDeltaSlots][kDeltaFields]
    int32_t j;                    // step offset within the launch sequence
    int32_t n;
    // push form of the pressure (fs_push.cu): per-node infectious in-neighbour
    // counts kept up to date by +-1 pushes along the transposed CSR; pushes
    // made at step k land in the pending words of parity k & 1
    uint8_t* cnt8;                // [n_thr] counts of the thread class (in-degree <= 255)
    uint16_t* pd16[2];            // [n_thr] pending pushes: +1 tally low byte, -1 tally high byte
    uint32_t* hcnt;               // [n_m] counts of the merge class
    unsigned long long* pd64[2];  // [n_m] pending pushes: +1 tally low word, -1 tally high word
    const int64_t* out_ptr;       // [n + 1] transposed CSR: the nodes whose rows list node j
    const int32_t* out_col;       // [nnz] internal ids
    // adaptive step (push kernel's ADAPTIVE instance): dt_k = min(M.dt,
    // eps / (lambda*_{k-1} + delta)); the size of step j of a launch
    // sequence is recorded in dtrec[j] for the epilogue's clock
    float eps, delta;
    float* dtrec;                 // [kMaxGraphSteps]
    // source-node infectivity with a shedding profile (Eq. 8; gather kernels'
    // SHED instances): rho[k & 1][i] = beta s(tau_i) of the nodes that are I
    // at step k, in the storage type of the ages; entries of other nodes are
    // stale and never read (the bitmap gates every read)
    void* rho[2];
    float2* m_part;               // [n_chunks] cross-chunk partial pressures: .x of the row that
                                  // enters the chunk from the previous one, .y of the row that
                                  // continues into the next one
    LawF shed;                    // the law of s(tau)
    int32_t shed_mode;            // FS_SHED_HAZARD (1) or FS_SHED_DENSITY (2); 0 = s = 1
    const float4* rtab;           // [kPTableN] memoised beta s(age) over the fixed-step age
                                  // sequence, two (age, value) slots per index like ptab
    // active-node compaction (null: off): the units with a non-R node at the
    // start of the launch sequence, ctl->n_act of them (all units when
    // n_act >= their number): SELL slices (gather) or push items
    int32_t* act;
    // Markovian engine (fs_markov.cu): exact infectious in-neighbour counts of
    // every node, the step's event list, the rates and the step-size rule
    uint32_t* mk_cnt;             // [n]
    uint32_t* mk_ev;              // [n] node | bit 31 when it left I
    double mk_beta, mk_sigma, mk_gamma;
    double mk_theta, mk_p_max, mk_tau_max;
    double mk_avg_deg;            // edges / nodes
    int64_t e_total;              // edges
    int32_t mk_mode;              // influence update: 0 by cost, 1 inertial, 2 control
    // failure-detection tests (fs_test_inject): the bounded mbarrier waits
    // give up after wait_limit polls (0 = kWaitLimit); with skip_bulk_copy
    // set the merge chunks arm their barrier but issue no copy, so their
    // waits run out with nothing in flight
    uint32_t wait_limit;
    int32_t skip_bulk_copy;
    // lengths the FS_DEBUG_BOUNDS checks compare against (set in every
    // build; read only by bounds-checked builds): node slots of X, entries
    // of the transposed CSR (minus dbg_shrink, a test knob that puts the
    // check's bound below the buffer's end), SELL column entries, bitmap words
    int64_t x_len;
    int64_t out_nnz;
    int64_t dbg_shrink;
    int64_t sell_len;
    int64_t bm_words;
};

enum { kShedNone = 0, kShedHazard = 1, kShedDensity = 2 };

constexpr int kPushG = 8;                 // thread-class nodes per thread of the push step
// 128-thread CTAs: at N = 10^6 the one-item-per-lane grid has ~7 CTAs per
// SM rather than ~3, so the epidemic peak (issue-bound per SM) is spread more
// evenly over the SMs (measured 6.65 vs 6.92 us per step against 256)
constexpr int kPushThreads = 128;                      // threads per CTA of the push step
constexpr int kPushCtasPerSm = 1024 / kPushThreads;    // resident CTAs per SM (64 registers a thread)

}  // namespace fs

namespace fs {

// ---------------------------------------------------------------------------
// Packed ensembles: up to 32 realisations of one graph stored node-major
// (state[i * R_pad + r]), stepped together so that one column read serves
// every replicate. A batch steps many such segments in one launch per step
// through a device segment table.
// ---------------------------------------------------------------------------
constexpr int kPackMaxR = 32;
constexpr int kPackClasses = 18;        // 3 replicate widths x 3 pressure forms x 2 step rules
constexpr int kPackThreads = 128;       // threads per block of the packed step

struct __align__(16) PackScen {   // one realisation of a segment
    // what the step reads per replicate, as three 16-byte words
    const float4* ptab;     // [2][kPTableN] memoised probabilities of its laws (two slots per index)
    const float* ps;        // [kPSTableN]
    uint32_t key0, key1, rep;   // copies of M.key0, M.key1, M.rep (Philox key and replicate index)
    float dt;               // copy of M.dt
    float beta, inv_dt;     // copies of M.beta, M.inv_dt
    float eps, delta;       // adaptive step (eps > 0): dt_k = min(dt, eps / (lambda*_{k-1} + delta))
    ModelF M;               // all parameters (direct evaluation when a table misses)
    // shedding profile (Section 5.3, Eq. 8; segments with shed != 0):
    // rtab[kPTableN] memoises beta s(age) over the fixed-step age sequence
    const float4* rtab;
    LawF shed;
    int32_t shed_mode;
    int32_t pad_;
};

struct PackSeg {            // one row of the segment table
    // graph in internal node order (shared with single-realisation sims)
    const int64_t* sell_off;
    const int32_t* sell_col;
    const int64_t* m_ptr;   // merge-class (hub) rows, relative to m_base = n_thr
    const int32_t* m_col;
    const int32_t* perm;    // internal -> original id (null = identity)
    int32_t n, n_thr, n_slices, n_m, sentinel;
    int32_t R_pad;          // 8, 16 or 32 lanes per node
    int32_t R;              // live realisations (r >= R are inert padding, state R)
    int32_t model;
    // packed state
    uint8_t* X;             // [n][R_pad]
    void* A;                // [n][R_pad] ages of the batch's storage type
    void* mask[2];          // [n + 1] R_pad-bit infectious masks by local step parity
    const PackScen* scen;   // [R_pad]
    int64_t join;           // the segment's step index at global step G is k = G - join
    int64_t kmin, kend;     // it runs steps kmin .. kend-1; counts row k - kmin after step k-1
    unsigned long long* deltas;   // [2][R_pad][3] per-replicate transitions by local step parity
    uint32_t* counts;       // [R_pad][4] running counts
    uint32_t* out;          // [(steps + 1)][R_pad][4] counts after each step, or null
    // push form of the pressure (push != 0; the masks above are then unused):
    // per (node, replicate) infectious in-neighbour counts and pending +1/-1
    // tallies by local step parity, laid out like X, and the transposed CSR
    int32_t push;
    int32_t pad2_;
    uint8_t* pc8;                   // [n_thr][R_pad] counts of the thread class
    uint16_t* ppd[2];               // [n_thr][R_pad] tallies: +1 low byte, -1 high byte
    uint32_t* phc;                  // [n_m][R_pad] counts of merge-class nodes
    unsigned long long* phpd[2];    // [n_m][R_pad] tallies: +1 low word, -1 high word
    const int64_t* out_ptr;         // [n + 1]
    const int32_t* out_col;         // [nnz]
    // adaptive step (every realisation of the segment has eps > 0; null =
    // fixed step): lam[(k % 3) * R_pad + r] = the largest rate of replicate r
    // in step k (FP32 bits, atomic max); step k reads slot (k + 2) % 3 for its
    // size, the launch of step k clears slot (k + 1) % 3; time[r] = replicate
    // r's simulated clock
    uint32_t* lam;
    double* time;
    // shedding profile (gather form; shed != 0): rho[par][i * R_pad + r] =
    // beta s(tau) of replicate r of node i while it is I (storage type of the
    // ages; read only where the infectious mask has the replicate's bit), by
    // local step parity; S replicates sum the rho of their infectious
    // in-neighbours in FP32
    void* rho[2];
    int32_t shed;
    int32_t pad3_;
};

// The segment table is ordered by replicate width (R_pad 8, 16, 32); each
// width is stepped by its own kernel instance, whose register budget suits it.
struct PackArgs {
    const PackSeg* seg;       // segment table
    const int64_t* thr_pre;   // [n_seg + 1] exclusive prefix of SELL work items
    const int64_t* hub_pre;   // [n_seg + 1] exclusive prefix of hub rows
    const int32_t* cls;       // [kPackClasses + 1] rows [cls[i], cls[i+1]) with i = (3c + f) * 2 + d have
                              // R_pad = 8 << c, pressure form f (0 gather, 1 push, 2 gather with a
                              // shedding profile) and step d (0 fixed, 1 adaptive)
                              // (device, updated between launches)
    DevCtl* ctl;              // global step counter and error word
    int32_t j;                // step offset within the launch sequence
};

}  // namespace fs
