// fs_ingest.cu -- graph ingest on the device: degrees and the degree
// profile (Section 5.5: one pass over row_ptr gives d_max and rho), a stable
// counting sort of the nodes by degree class, the SELL-32 column blocks of
// the one-thread-per-node class, and the CSR and chunk tables of the
// edge-partitioned merge class (Appendix B.3 merge-path partition).
#include <cuda_runtime.h>

#include <climits>

#include "fs_launch.h"

namespace fs {

constexpr uint32_t kFullMask = 0xffffffffu;

// deg[i] = row_ptr[i+1] - row_ptr[i]; key = deg if deg <= t1 else t1 + 1.
// Also: d_max, count of deg <= t1, monotonicity of row_ptr, and whether the
// keys are already nondecreasing (then no relabelling is needed).
__global__ void degree_kernel(const int64_t* __restrict__ row_ptr, int n, int t1, int32_t* __restrict__ deg,
                              uint16_t* __restrict__ key, IngestFlags* flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int d = 0, k = 0, bad = 0, small = 0;
    if (i < n) {
        const int64_t a = row_ptr[i], b = row_ptr[i + 1];
        const int64_t dd = b - a;
        if (dd < 0 || dd > INT_MAX || (i == 0 && a != 0))
            bad = 1;
        d = (int)max((int64_t)0, min(dd, (int64_t)INT_MAX));
        k = d <= t1 ? d : t1 + 1;
        small = d <= t1;
        if (deg) {                                   // null: only d_max and the checks
            deg[i] = d;
            key[i] = (uint16_t)k;
        }
        if (i + 1 < n) {
            const int64_t dn = row_ptr[i + 2] - b;
            const int kn = (dn >= 0 && dn <= t1) ? (int)dn : t1 + 1;
            if (kn < k)
                atomicOr(&flags->unsorted, 1);
        }
    }
    int m = d;
    for (int o = 16; o > 0; o >>= 1)
        m = max(m, __shfl_xor_sync(kFullMask, m, o));
    const int cs = __popc(__ballot_sync(kFullMask, small));
    const int anybad = __any_sync(kFullMask, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&flags->dmax, m);
        if (cs)
            atomicAdd(&flags->n_thr, cs);
        if (anybad)
            atomicOr(&flags->error, 1);
    }
}

__global__ void check_cols_kernel(const int32_t* __restrict__ col, int64_t nnz, int n, IngestFlags* flags)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool bad = e < nnz && (col[e] < 0 || col[e] >= n);
    if (__any_sync(kFullMask, bad) && (threadIdx.x & 31) == 0)
        atomicOr(&flags->error, 2);
}

// --- stable counting sort ---------------------------------------------------
// Tile = 256 consecutive nodes (8 warps). Within a warp the stable rank of a
// node among equal keys comes from __match_any_sync; across the tile's warps
// a per-warp histogram in shared memory adds the earlier warps' counts. The
// per-(bucket, tile) counts are scanned bucket-major, which gives every node
// its final position.
constexpr int kSortTile = 256;

template <bool SCATTER>
__global__ void __launch_bounds__(kSortTile) sort_tile_kernel(const uint16_t* __restrict__ key,
                                                              const int32_t* __restrict__ deg, int n,
                                                              int n_buckets, int n_tiles,
                                                              int64_t* __restrict__ counts,
                                                              int32_t* __restrict__ perm, int32_t* __restrict__ inv,
                                                              int32_t* __restrict__ deg_int)
{
    extern __shared__ int32_t whist[];   // [8][n_buckets]
    const int tile = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < 8 * n_buckets; t += blockDim.x)
        whist[t] = 0;
    __syncthreads();
    const int i = tile * kSortTile + threadIdx.x;
    const bool valid = i < n;
    const int k = valid ? (int)key[i] : n_buckets;   // invalid lanes form their own group
    const uint32_t peers = __match_any_sync(kFullMask, k);
    const int rank_w = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank_w == 0)
        whist[warp * n_buckets + k] = __popc(peers);
    __syncthreads();
    if (!SCATTER) {
        for (int b = threadIdx.x; b < n_buckets; b += blockDim.x) {
            int64_t s = 0;
            for (int w = 0; w < 8; ++w)
                s += whist[w * n_buckets + b];
            counts[(int64_t)b * n_tiles + tile] = s;
        }
    } else if (valid) {
        int64_t pos = counts[(int64_t)k * n_tiles + tile] + rank_w;
        for (int w = 0; w < warp; ++w)
            pos += whist[w * n_buckets + k];
        perm[pos] = i;
        inv[i] = (int32_t)pos;
        deg_int[pos] = deg[i];
    }
}

// --- exclusive scan of int64 ------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;   // 2048 elements per block

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total)
{
    __shared__ int64_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFullMask, w, o);
            if (lane >= o)
                w += y;
        }
        if (lane < kScanThreads / 32)
            warp_sums[lane] = w;
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void scan_reduce_kernel(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    int64_t s = 0;
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t i = base + (int64_t)t * kScanThreads + threadIdx.x;
        if (i < n)
            s += in[i];
    }
    int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0)
        sums[blockIdx.x] = tot;
}

// out[i] = offset[block] + exclusive sum within the block; the last block
// also writes out[n] when write_total is set
__global__ void scan_apply_kernel(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ offsets,
                                  int64_t* __restrict__ out)
{
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanItems + t;
        v[t] = (i < n) ? in[i] : 0;
        s += v[t];
    }
    int64_t tot;
    int64_t run = block_exclusive_scan(s, &tot) + (offsets ? offsets[blockIdx.x] : 0);
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanItems + t;
        if (i < n)
            out[i] = run;
        run += v[t];
        if (i == n - 1)
            out[n] = run;
    }
}

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s)
{
    if (n <= 0)
        return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    const int64_t blocks = (n + kScanBlock - 1) / kScanBlock;
    if (blocks == 1) {
        scan_apply_kernel<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        g_launch_count += 1;
        return cudaGetLastError();
    }
    int64_t* sums = nullptr;
    cudaError_t e = cudaMallocAsync(&sums, sizeof(int64_t) * (blocks + 1), s);
    if (e != cudaSuccess)
        return e;
    scan_reduce_kernel<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, n, sums);
    g_launch_count += 2;
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = exclusive_scan_i64(sums, sums, blocks, s);   // in place: each block reads before writing
    if (e == cudaSuccess) {
        scan_apply_kernel<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, n, sums, out);
        e = cudaGetLastError();
    }
    cudaFreeAsync(sums, s);
    return e;
}

cudaError_t stable_sort_by_key(const uint16_t* key, const int32_t* deg, int n, int n_buckets, int32_t* perm,
                               int32_t* inv, int32_t* deg_int, cudaStream_t s)
{
    const int n_tiles = (n + kSortTile - 1) / kSortTile;
    const int64_t m = (int64_t)n_buckets * n_tiles;
    int64_t* counts = nullptr;
    cudaError_t e = cudaMallocAsync(&counts, sizeof(int64_t) * (m + 1), s);
    if (e != cudaSuccess)
        return e;
    const size_t smem = sizeof(int32_t) * 8 * n_buckets;
    sort_tile_kernel<false><<<n_tiles, kSortTile, smem, s>>>(key, deg, n, n_buckets, n_tiles, counts, nullptr,
                                                             nullptr, nullptr);
    g_launch_count += 2;
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = exclusive_scan_i64(counts, counts, m, s);
    if (e == cudaSuccess) {
        sort_tile_kernel<true><<<n_tiles, kSortTile, smem, s>>>(key, deg, n, n_buckets, n_tiles, counts, perm, inv,
                                                                deg_int);
        e = cudaGetLastError();
    }
    cudaFreeAsync(counts, s);
    return e;
}

// --- SELL-32 of the thread class ---------------------------------------------
__global__ void sell_width_kernel(const int32_t* __restrict__ deg_int, int n_thr, int n_slices,
                                  int64_t* __restrict__ width32)
{
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int i = w * 32 + lane;
    int d = (w < n_slices && i < n_thr) ? deg_int[i] : 0;
    for (int o = 16; o > 0; o >>= 1)
        d = max(d, __shfl_xor_sync(kFullMask, d, o));
    if (lane == 0 && w < n_slices)
        width32[w] = (int64_t)d * 32;
}

// one warp per slice: column t of lane j at sell_off[s] + 32 t + j
__global__ void sell_fill_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                                 const int32_t* __restrict__ deg_int, int n_thr, int n_slices,
                                 const int64_t* __restrict__ sell_off, int sentinel, int32_t* __restrict__ sell_col)
{
    const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= n_slices)
        return;
    const int i = s * 32 + lane;
    const int64_t off = sell_off[s];
    const int w = (int)((sell_off[s + 1] - off) >> 5);
    int d = 0;
    int64_t rs = 0;
    if (i < n_thr) {
        const int o = perm ? perm[i] : i;
        d = deg_int[i];
        rs = row_ptr[o];
    }
    for (int t = 0; t < w; ++t) {
        int v = sentinel;
        if (t < d) {
            const int j = col[rs + t];
            v = inv ? inv[j] : j;
        }
        sell_col[off + 32 * (int64_t)t + lane] = v;
    }
}

// --- merge class ---------------------------------------------------------------
__global__ void merge_deg_kernel(const int32_t* __restrict__ deg_int, int m_base, int n_m, int64_t* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_m)
        out[r] = deg_int[m_base + r];
}

// one warp per row (coalesced), then the padding up to whole chunks
__global__ void merge_fill_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ perm, const int32_t* __restrict__ inv, int m_base,
                                  int n_m, const int64_t* __restrict__ m_ptr, int64_t e_m, int64_t padded,
                                  int sentinel, int32_t* __restrict__ m_col)
{
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw < n_m) {
        const int r = (int)gw;
        const int o = perm ? perm[m_base + r] : m_base + r;
        const int64_t src = row_ptr[o];
        const int64_t dst = m_ptr[r];
        const int64_t d = m_ptr[r + 1] - dst;
        for (int64_t t = lane; t < d; t += 32) {
            const int j = col[src + t];
            m_col[dst + t] = inv ? inv[j] : j;
        }
    } else {
        const int64_t p = e_m + (gw - n_m) * 32 + lane;
        if (p < padded)
            m_col[p] = sentinel;
    }
}

// row r with m_ptr[r] <= e < m_ptr[r+1] (rows have degree >= 1)
__device__ __forceinline__ int row_of_edge(const int64_t* m_ptr, int n_m, int64_t e)
{
    int lo = 0, hi = n_m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m_ptr[mid] <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void merge_table_kernel(const int64_t* __restrict__ m_ptr, int n_m, int64_t e_m, int n_chunks,
                                   int32_t* __restrict__ warp_row, int32_t* __restrict__ chunk_last)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n_w = (int64_t)n_chunks * kStepWarps;
    if (t < n_w) {
        const int64_t e = t * kMergeEdgesPerWarp;
        warp_row[t] = row_of_edge(m_ptr, n_m, min(e, e_m - 1));
    }
    if (t < n_chunks) {
        const int64_t last = min((t + 1) * (int64_t)kMergeEPB, e_m) - 1;
        chunk_last[t] = row_of_edge(m_ptr, n_m, last);
    }
}

// --- launchers -----------------------------------------------------------------
cudaError_t launch_degrees(const int64_t* row_ptr, int n, int t1, int32_t* deg, uint16_t* key, IngestFlags* flags,
                           cudaStream_t s)
{
    degree_kernel<<<(n + 255) / 256, 256, 0, s>>>(row_ptr, n, t1, deg, key, flags);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_check_cols(const int32_t* col, int64_t nnz, int n, IngestFlags* flags, cudaStream_t s)
{
    if (nnz == 0)
        return cudaSuccess;
    check_cols_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(col, nnz, n, flags);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_sell_widths(const int32_t* deg_int, int n_thr, int n_slices, int64_t* width32, cudaStream_t s)
{
    if (n_slices == 0)
        return cudaSuccess;
    const int64_t threads = (int64_t)n_slices * 32;
    sell_width_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(deg_int, n_thr, n_slices, width32);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_sell_fill(const int64_t* row_ptr, const int32_t* col, const int32_t* perm, const int32_t* inv,
                             const int32_t* deg_int, int n_thr, int n_slices, const int64_t* sell_off, int sentinel,
                             int32_t* sell_col, cudaStream_t s)
{
    if (n_slices == 0)
        return cudaSuccess;
    const int64_t threads = (int64_t)n_slices * 32;
    sell_fill_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(row_ptr, col, perm, inv, deg_int, n_thr,
                                                                       n_slices, sell_off, sentinel, sell_col);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_merge_degrees(const int32_t* deg_int, int m_base, int n_m, int64_t* out, cudaStream_t s)
{
    if (n_m == 0)
        return cudaSuccess;
    merge_deg_kernel<<<(n_m + 255) / 256, 256, 0, s>>>(deg_int, m_base, n_m, out);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_merge_fill(const int64_t* row_ptr, const int32_t* col, const int32_t* perm, const int32_t* inv,
                              int m_base, int n_m, const int64_t* m_ptr, int64_t e_m, int64_t padded, int sentinel,
                              int32_t* m_col, cudaStream_t s)
{
    const int64_t warps = (int64_t)n_m + (padded - e_m + 31) / 32;
    if (warps == 0)
        return cudaSuccess;
    merge_fill_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(row_ptr, col, perm, inv, m_base, n_m,
                                                                           m_ptr, e_m, padded, sentinel, m_col);
    g_launch_count += 1;
    return cudaGetLastError();
}

cudaError_t launch_merge_tables(const int64_t* m_ptr, int n_m, int64_t e_m, int n_chunks, int32_t* warp_row,
                                int32_t* chunk_last, cudaStream_t s)
{
    const int64_t t = (int64_t)n_chunks * kStepWarps;
    if (t == 0)
        return cudaSuccess;
    merge_table_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(m_ptr, n_m, e_m, n_chunks, warp_row, chunk_last);
    g_launch_count += 1;
    return cudaGetLastError();
}

}  // namespace fs
