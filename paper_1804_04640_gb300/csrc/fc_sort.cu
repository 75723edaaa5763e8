// fc_sort.cu -- counting by sorting, for tables too large for shared memory.
//
// Sec. 3.3 partitions the instances by the states of the query variables,
// most significant digit first (Alg. 2-3); the partition sizes are the
// counts.  Here the partitions are found by sorting instead of recursive
// bucketing: each instance gets its mixed-radix key (its cell index, the
// parents' digits most significant and the child's least, as in Sec. 3.3),
// the keys are sorted with a stable least-significant-digit radix sort
// (8-bit digits, only as many passes as the key has bits), and every run of
// equal keys is one non-empty partition whose length is the count.
//
// Run lengths are written without a search for run ends: the first element
// of a run at position p adds -p to its cell and the last element at position
// p' adds p' + 1, so a zeroed cell ends up holding the run length.
#include "fc_internal.h"

#include <mutex>

#include "../../include/fc.h"

// Scratch of the allocation-free entry point fc_count_sorted_noalloc: two key
// buffers and the per-tile digit histograms of the radix sort, sized for at
// most 2^20 instances (8.25 MiB).  Every GPU that loads the library holds it
// until the process exits.  Host code must not use this name as an address:
// the device address comes from cudaGetSymbolAddress (see below).
static __device__ __align__(256) uint32_t g_noalloc_scratch[2 * (1 << 20) + 256 * ((1 << 20) / 4096)];

namespace fc {
namespace {

constexpr int kTile = 4096;     // keys per block of the radix passes
constexpr int kThreads = 256;   // 8 warps, 512 keys each
constexpr int kWarps = kThreads / 32;
constexpr int kPerWarp = kTile / kWarps;

__global__ void keys_kernel(const uint8_t *__restrict__ D, int64_t m_pad, int64_t m,
                            const QVar *__restrict__ vars, int32_t k, uint32_t *keys)
{
    __shared__ QVar s_vars[kMaxK];
    if (threadIdx.x < k) s_vars[threadIdx.x] = vars[threadIdx.x];
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t key = 0u;
        for (int t = 0; t < k; ++t)
            key += (uint32_t)D[(int64_t)s_vars[t].var * m_pad + p] * (uint32_t)s_vars[t].stride;
        keys[p] = key;
    }
}

// Digit histogram of one tile: hist[d * nblocks + block].
__global__ void digit_hist_kernel(const uint32_t *__restrict__ keys, int64_t m, int shift,
                                  uint32_t *hist, int nblocks)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        const int64_t p = base + i;
        if (p < m) atomicAdd(&h[(keys[p] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of n entries in one block of 1024 threads.
__global__ void exclusive_scan_kernel(uint32_t *a, int64_t n)
{
    __shared__ uint32_t warp_sums[32];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * per;
    const int64_t hi = min(n, lo + per);
    uint32_t sum = 0u;
    for (int64_t i = lo; i < hi; ++i) sum += a[i];
    // block exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t run = incl - sum + (warp > 0 ? warp_sums[warp - 1] : 0u);
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// Stable scatter of one tile.  Warp w owns keys [w * 512, (w + 1) * 512) of the
// tile and walks them in order, 32 at a time; lanes holding the same digit
// rank themselves with __match_any_sync, so equal digits keep their order.
__global__ void scatter_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                               int64_t m, int shift, const uint32_t *__restrict__ offs,
                               int nblocks)
{
    __shared__ uint32_t whist[kWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kWarps * 256; d += kThreads) (&whist[0][0])[d] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * kPerWarp;
    for (int i = lane; i < kPerWarp; i += 32) {
        const int64_t p = base + i;
        if (p < m) atomicAdd(&whist[warp][(in[p] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // kThreads == 256 digits
        uint32_t run = offs[(int64_t)d * nblocks + blockIdx.x];
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = whist[w][d];
            whist[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int i = 0; i < kPerWarp; i += 32) {
        const int64_t p = base + i + lane;
        const bool ok = p < m;
        const uint32_t key = ok ? in[p] : 0u;
        const uint32_t d = ok ? ((key >> shift) & 0xffu) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt);
        const uint32_t pos = ok ? whist[warp][d] + rank : 0u;
        __syncwarp();
        if (ok) {
            out[pos] = key;
            if (rank == (unsigned)__popc(peers) - 1u) whist[warp][d] += (uint32_t)__popc(peers);
        }
        __syncwarp();
    }
}

// A key that occurs in several runs (possible only for keys outside the
// table, see keys_byval_kernel) still adds up to its count: every run adds
// its own length.  Keys >= cells are not counted.
__global__ void run_length_kernel(const uint32_t *__restrict__ sorted, int64_t m, int32_t *table,
                                  uint32_t cells)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = sorted[p];
        if (key >= cells) continue;
        if (p == 0 || sorted[p - 1] != key) atomicAdd(&table[key], (int32_t)(-p));
        if (p == m - 1 || sorted[p + 1] != key) atomicAdd(&table[key], (int32_t)(p + 1));
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > 4096) g = 4096;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int sort_tile_rows() { return kTile; }

cudaError_t launch_sort_count(const uint8_t *D, int64_t m_pad, int64_t m, const QVar *d_vars,
                              int32_t k, int32_t key_bits, int32_t *table, int32_t cells,
                              int32_t zero_table, SortScratch sc, cudaStream_t s)
{
    cudaError_t e;
    if (zero_table) {
        e = cudaMemsetAsync(table, 0, (size_t)cells * sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
    }
    if (m <= 0) return cudaSuccess;
    const int nblocks = (int)((m + kTile - 1) / kTile);
    if (m > sc.cap_rows || nblocks > sc.cap_blocks) return cudaErrorInvalidValue;
    keys_kernel<<<grid_for(m, 256), 256, 0, s>>>(D, m_pad, m, d_vars, k, sc.keys_a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uint32_t *a = sc.keys_a, *b = sc.keys_b;
    for (int shift = 0; shift < key_bits; shift += 8) {
        digit_hist_kernel<<<nblocks, kThreads, 0, s>>>(a, m, shift, sc.block_hist, nblocks);
        exclusive_scan_kernel<<<1, 1024, 0, s>>>(sc.block_hist, (int64_t)nblocks * 256);
        scatter_kernel<<<nblocks, kThreads, 0, s>>>(a, b, m, shift, sc.block_hist, nblocks);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint32_t *t = a;
        a = b;
        b = t;
    }
    run_length_kernel<<<grid_for(m, 256), 256, 0, s>>>(a, m, table, (uint32_t)cells);
    return cudaGetLastError();
}


// ------------------------------------------------- allocation-free variant

namespace {

constexpr int64_t kNoAllocMaxRows = (int64_t)1 << 20;
constexpr int kNoAllocMaxDevices = 64;

struct KeyDesc {
    int32_t k;
    QVar v[kMaxK];
};

// Keys with the descriptors passed by value (no device-side descriptor
// buffer).  An instance whose state is outside its variable's arity gets the
// key 0xFFFFFFFF and is not counted.
__global__ void keys_byval_kernel(const uint8_t *__restrict__ D, int64_t ld, int64_t m, const KeyDesc d,
                                  uint32_t *keys)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t key = 0u;
        bool bad = false;
        for (int t = 0; t < d.k; ++t) {
            const uint32_t st = D[(int64_t)d.v[t].var * ld + p];
            bad |= st >= (uint32_t)d.v[t].arity;
            key += st * (uint32_t)d.v[t].stride;
        }
        keys[p] = bad ? 0xFFFFFFFFu : key;
    }
}

std::mutex g_noalloc_mu;
uint32_t *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the lookup allocates nothing).
cudaError_t noalloc_scratch(int dev, uint32_t **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (uint32_t *)p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace fc

extern "C" int fc_count_sorted_noalloc(const uint8_t *D, int32_t n, int64_t m, int64_t ld,
                                       const int32_t *arities, const int32_t *vars, int32_t k,
                                       int32_t *table, void *stream)
{
    using namespace fc;
    if ((!D && m > 0) || !arities || !table || (k > 0 && !vars))
        return set_error(FC_ERR_ARG, "fc_count_sorted_noalloc: null argument");
    if (n < 1 || m < 0 || ld < m || k < 0 || k > kMaxK)
        return set_error(FC_ERR_ARG, "fc_count_sorted_noalloc: bad n, m, ld or k");
    if (m > kNoAllocMaxRows)
        return set_error(FC_ERR_SIZE, "fc_count_sorted_noalloc counts at most %lld instances, got %lld",
                         (long long)kNoAllocMaxRows, (long long)m);
    KeyDesc d{};
    d.k = k;
    int64_t cells = 1;
    for (int t = 0; t < k; ++t) {
        const int v = vars[t];
        if (v < 0 || v >= n) return set_error(FC_ERR_ARG, "variable %d out of range", v);
        for (int u = 0; u < t; ++u)
            if (vars[u] == v) return set_error(FC_ERR_ARG, "variable %d listed twice", v);
        if (arities[v] < 1 || arities[v] > 255) return set_error(FC_ERR_ARG, "arity of variable %d not in 1..255", v);
        cells *= arities[v];
        if (cells > INT32_MAX) return set_error(FC_ERR_SIZE, "table exceeds 2^31-1 cells");
    }
    int64_t stride = 1;
    for (int t = k - 1; t >= 0; --t) {
        d.v[t] = QVar{vars[t], (int32_t)stride, arities[vars[t]], 0};
        stride *= arities[vars[t]];
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return set_error(FC_ERR_CUDA, "fc_count_sorted_noalloc: no usable current device");
    uint32_t *scratch = nullptr;
    if ((e = noalloc_scratch(dev, &scratch)) != cudaSuccess)
        return set_error(FC_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    if ((e = cudaMemsetAsync(table, 0, (size_t)cells * sizeof(int32_t), s)) != cudaSuccess)
        return set_error(FC_ERR_CUDA, "zeroing the table: %s", cudaGetErrorString(e));
    if (m == 0) return FC_OK;
    const int nblocks = (int)((m + kTile - 1) / kTile);
    uint32_t *a = scratch, *b = scratch + kNoAllocMaxRows, *hist = scratch + 2 * kNoAllocMaxRows;
    const int key_bits = cells > 1 ? 32 - __builtin_clz((uint32_t)(cells - 1)) : 0;
    keys_byval_kernel<<<grid_for(m, 256), 256, 0, s>>>(D, ld, m, d, a);
    for (int shift = 0; shift < key_bits; shift += 8) {
        digit_hist_kernel<<<nblocks, kThreads, 0, s>>>(a, m, shift, hist, nblocks);
        exclusive_scan_kernel<<<1, 1024, 0, s>>>(hist, (int64_t)nblocks * 256);
        scatter_kernel<<<nblocks, kThreads, 0, s>>>(a, b, m, shift, hist, nblocks);
        uint32_t *t = a;
        a = b;
        b = t;
    }
    run_length_kernel<<<grid_for(m, 256), 256, 0, s>>>(a, m, table, (uint32_t)cells);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return set_error(FC_ERR_CUDA, "fc_count_sorted_noalloc launch: %s", cudaGetErrorString(e));
    return FC_OK;
}
