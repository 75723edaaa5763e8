// fc_pack.cu -- load-time layout kernels: column-major database, per-state
// bitmaps (Sec. 3.2, Fig. 1a: one bitmap of m bits per state of each
// variable), marginal popcounts, and the specific-assignment count (the
// single root-to-leaf path of Alg. 1, end of Sec. 3.3).
#include "fc_internal.h"

namespace fc {
namespace {

// One warp packs 64 consecutive instances of one variable: for every state s
// the two ballots over (D_i[p] == s) are the low and high halves of word
// p / 64 of bitmap (i, s).  A state >= r_i sets *bad_state.
__global__ void pack_bits_kernel(const uint8_t *__restrict__ D, int64_t m_pad, int64_t m,
                                 const int32_t *__restrict__ arity,
                                 const int32_t *__restrict__ soff, uint64_t *__restrict__ bits,
                                 int64_t wstride, int32_t *bad_state)
{
    const int i = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w * 64 >= m) return;  // whole warp leaves together
    const int64_t p0 = w * 64 + lane, p1 = p0 + 32;
    const uint8_t *col = D + (int64_t)i * m_pad;
    const int r = arity[i];
    const int b0 = p0 < m ? (int)col[p0] : -1;
    const int b1 = p1 < m ? (int)col[p1] : -1;
    if (b0 >= r || b1 >= r) atomicOr(bad_state, 1);
    uint64_t *row = bits + (int64_t)soff[i] * wstride + w;
    for (int s = 0; s < r; ++s) {
        const unsigned lo = __ballot_sync(0xffffffffu, b0 == s);
        const unsigned hi = __ballot_sync(0xffffffffu, b1 == s);
        if (lane == (s & 31)) row[(int64_t)s * wstride] = ((uint64_t)hi << 32) | lo;
    }
}

__global__ void bit_popcount_kernel(const uint64_t *__restrict__ bits, int64_t wstride,
                                    int64_t *counts)
{
    const uint64_t *row = bits + (int64_t)blockIdx.x * wstride;
    unsigned long long c = 0;
    for (int64_t w = threadIdx.x; w < wstride; w += blockDim.x) c += __popcll(row[w]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned long long part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += part[j];
        counts[blockIdx.x] = (int64_t)t;
    }
}

// Row-major (m x n) -> column-major (n x m_pad) through a 32 x 32 byte tile.
__global__ void transpose_rows_kernel(const uint8_t *__restrict__ Drow, int64_t m, int32_t n,
                                      uint8_t *__restrict__ Dcol, int64_t m_pad)
{
    __shared__ uint8_t tile[32][33];
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    const int i0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t p = p0 + dy;
        const int i = i0 + threadIdx.x;
        if (p < m && i < n) tile[dy][threadIdx.x] = Drow[p * n + i];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int i = i0 + dy;
        const int64_t p = p0 + threadIdx.x;
        if (p < m && i < n) Dcol[(int64_t)i * m_pad + p] = tile[threadIdx.x][dy];
    }
}

__global__ void mask_tail_kernel(uint64_t *bits, int64_t wstride, int64_t m)
{
    uint64_t *row = bits + (int64_t)blockIdx.x * wstride;
    const int64_t full = m / 64;
    for (int64_t w = full + threadIdx.x; w < wstride; w += blockDim.x) {
        if (w == full && (m % 64) != 0)
            row[w] &= (~0ull) >> (64 - (m % 64));
        else
            row[w] = 0ull;
    }
}

__global__ void assignment_count_kernel(const uint64_t *__restrict__ bits, int64_t wstride,
                                        const int32_t *__restrict__ rows, int32_t k,
                                        int64_t words, unsigned long long *out)
{
    unsigned long long c = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = ~0ull;
        for (int t = 0; t < k; ++t) x &= bits[(int64_t)rows[t] * wstride + w];
        c += __popcll(x);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace

cudaError_t launch_pack_bits(const uint8_t *D, int64_t m_pad, int64_t m, int32_t n,
                             const int32_t *d_arity, const int32_t *d_soff, uint64_t *bits,
                             int64_t wstride, int32_t /*max_arity*/, int32_t *bad_state,
                             cudaStream_t s)
{
    const int warps = 8;
    const int64_t words = (m + 63) / 64;
    dim3 grid((unsigned)((words + warps - 1) / warps), (unsigned)n);
    pack_bits_kernel<<<grid, warps * 32, 0, s>>>(D, m_pad, m, d_arity, d_soff, bits, wstride,
                                                 bad_state);
    return cudaGetLastError();
}

cudaError_t launch_bit_popcounts(const uint64_t *bits, int64_t rows, int64_t wstride,
                                 int64_t *counts, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    bit_popcount_kernel<<<(unsigned)rows, 256, 0, s>>>(bits, wstride, counts);
    return cudaGetLastError();
}

cudaError_t launch_transpose_rows(const uint8_t *Drow, int64_t m, int32_t n, uint8_t *Dcol,
                                  int64_t m_pad, cudaStream_t s)
{
    dim3 grid((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32));
    transpose_rows_kernel<<<grid, dim3(32, 8), 0, s>>>(Drow, m, n, Dcol, m_pad);
    return cudaGetLastError();
}

cudaError_t launch_mask_tail_bits(uint64_t *bits, int64_t rows, int64_t wstride, int64_t m,
                                  cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    mask_tail_kernel<<<(unsigned)rows, 128, 0, s>>>(bits, wstride, m);
    return cudaGetLastError();
}

cudaError_t launch_assignment_count(const uint64_t *bits, int64_t wstride, const int32_t *d_rows,
                                    int32_t k, int64_t words, unsigned long long *out,
                                    cudaStream_t s)
{
    int64_t blocks = (words + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    assignment_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(bits, wstride, d_rows, k, words, out);
    return cudaGetLastError();
}

}  // namespace fc
