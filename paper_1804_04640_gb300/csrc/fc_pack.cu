// fc_pack.cu -- load-time layout kernels: column-major database, per-state
// bitmaps (Sec. 3.2, Fig. 1a: one bitmap of m bits per state of each
// variable), marginal popcounts, and the specific-assignment count (the
// single root-to-leaf path of Alg. 1, end of Sec. 3.3).
#include "fc_internal.h"

#include <algorithm>

namespace fc {
namespace {

// One warp packs 32 consecutive words (2,048 instances) of one variable.  The
// warp first copies those 2 KiB of the column to shared memory with 16-byte
// loads.  In step j it reads instances 64 (w0 + j) + lane and + 32; ballots
// over them form word w0 + j, which lane j keeps, so after the 32 steps lane
// l holds word w0 + l and the stores are coalesced.
//
// Variables of at most 16 states are packed through bit planes: the ballots
// take bit k of each state (k < ceil(log2 r)), and each lane then forms every
// state's word as the AND of its planes or their complements, masked to the
// instances below m.  Larger arities take two ballots per state and step
// (states 16 at a time, a register per state and lane).
//
// A state >= r_i sets *bad_state (the caller then discards what was packed).
// With `delta` set, the bits of each state's words, except the `first_from`
// lowest bits of word first_word (instances that were there before), are
// added to delta[state]: the marginal counts of the packed instances.  The
// copy starts 64-byte aligned (m_pad is a multiple of 4096) and reads only
// vectors that start before m.
constexpr int kPackWarps = 8;
constexpr int kPlaneMaxArity = 16;
__global__ void __launch_bounds__(kPackWarps * 32) pack_bits_kernel(
    const uint8_t *__restrict__ D, int64_t m_pad, int64_t m, int64_t w0, const int32_t *__restrict__ arity,
    const int32_t *__restrict__ soff, uint64_t *__restrict__ bits, int64_t wstride, int32_t *bad_state,
    unsigned long long *delta, int first_from)
{
    __shared__ __align__(16) uint8_t s_rows[kPackWarps][2048];
    const int i = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wb = w0 + ((int64_t)blockIdx.x * kPackWarps + warp) * 32;
    const int64_t words = (m + 63) >> 6;
    if (wb >= words) return;  // whole warp leaves together
    const uint8_t *col = D + (int64_t)i * m_pad;
    const int r = arity[i];
    uint8_t *buf = s_rows[warp];
    {
        // only vectors that start before m: such a vector ends by
        // roundup(m, 16) <= m_pad, inside the column; instances past m are
        // never read back from the buffer
        const uint4 *src = reinterpret_cast<const uint4 *>(col + wb * 64);
        uint4 *dst = reinterpret_cast<uint4 *>(buf);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (wb * 64 + 16 * (lane + 32 * k) < m) dst[lane + 32 * k] = __ldg(src + lane + 32 * k);
    }
    __syncwarp();
    const int64_t my = wb + lane;  // the word this lane stores
    uint64_t *row = bits + (int64_t)soff[i] * wstride + my;
    const bool mine = my < words;
    // instances of my word that exist (below m) and that are counted in delta
    const int64_t left = m - 64 * my;
    const uint64_t valid = left >= 64 ? ~0ull : left > 0 ? (~0ull >> (64 - left)) : 0ull;
    const uint64_t counted = valid & ((my == w0 && first_from > 0) ? (~0ull << first_from) : ~0ull);
    auto emit = [&](int st, uint64_t w) {
        if (mine) row[(int64_t)st * wstride] = w;
        if (delta) {
            unsigned long long c = mine ? (unsigned long long)__popcll(w & counted) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0 && c) atomicAdd(delta + soff[i] + st, c);
        }
    };
    bool bad = false;
    if (r <= kPlaneMaxArity) {
        const int nb = r > 1 ? 32 - __clz(r - 1) : 1;  // bit planes of a state
        uint32_t plo[4] = {0u, 0u, 0u, 0u}, phi[4] = {0u, 0u, 0u, 0u};
        int top = 0;  // the largest state seen
        // step j: the ballots of bit k over instances 64 (wb + j) + lane and
        // + 32 are plane k of word wb + j; lane j keeps them
        auto step = [&](int j, int b0, int b1) {
            top = max(top, max(b0, b1));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k >= nb) break;
                const unsigned lo = __ballot_sync(0xffffffffu, b0 & (1 << k));
                const unsigned hi = __ballot_sync(0xffffffffu, b1 & (1 << k));
                if (lane == j) {
                    plo[k] = lo;
                    phi[k] = hi;
                }
            }
        };
        if ((wb + 32) * 64 <= m) {
            // every instance of the warp's 32 words exists
#pragma unroll 4
            for (int j = 0; j < 32; ++j) step(j, buf[j * 64 + lane], buf[j * 64 + 32 + lane]);
        } else {
            for (int j = 0; j < 32 && wb + j < words; ++j) {
                const int64_t p0 = (wb + j) * 64 + lane, p1 = p0 + 32;
                step(j, p0 < m ? (int)buf[j * 64 + lane] : 0, p1 < m ? (int)buf[j * 64 + 32 + lane] : 0);
            }
        }
        bad = top >= r;
        uint64_t plane[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) plane[k] = ((uint64_t)phi[k] << 32) | plo[k];
        for (int st = 0; st < r; ++st) {
            uint64_t w = valid;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < nb) w &= ((st >> k) & 1) ? plane[k] : ~plane[k];
            emit(st, w);
        }
    } else {
        for (int s0 = 0; s0 < r; s0 += 16) {
            uint64_t word[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) word[t] = 0ull;
            for (int j = 0; j < 32 && wb + j < words; ++j) {
                const int64_t p0 = (wb + j) * 64 + lane, p1 = p0 + 32;
                const int b0 = p0 < m ? (int)buf[j * 64 + lane] : -1;
                const int b1 = p1 < m ? (int)buf[j * 64 + 32 + lane] : -1;
                if (s0 == 0) bad |= (b0 >= r) | (b1 >= r);
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    if (s0 + t >= r) break;
                    const unsigned lo = __ballot_sync(0xffffffffu, b0 == s0 + t);
                    const unsigned hi = __ballot_sync(0xffffffffu, b1 == s0 + t);
                    if (lane == j) word[t] = ((uint64_t)hi << 32) | lo;
                }
            }
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (s0 + t < r) emit(s0 + t, word[t]);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(bad_state, 1);
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
// 4-bit state codes of column blockIdx.y: rows 2b and 2b + 1 in the low and
// high nibble of byte b, so a 32-bit word holds 8 consecutive rows in order.
// Each thread packs 16 rows (one 16-byte load, one 8-byte store) from row0 on.
__global__ void pack_codes4_kernel(const uint8_t *__restrict__ D, int64_t m_pad, int64_t row0, int64_t vecs,
                                   uint8_t *__restrict__ D4)
{
    const uint8_t *col = D + (int64_t)blockIdx.y * m_pad + row0;
    uint8_t *out = D4 + (int64_t)blockIdx.y * (m_pad / 2) + row0 / 2;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < vecs; v += (int64_t)gridDim.x * blockDim.x) {
        const uint4 x = *reinterpret_cast<const uint4 *>(col + v * 16);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
        uint32_t o[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            // bytes b0..b7 (states < 16) to nibbles n0..n7 of one word
            const uint32_t lo = w[2 * h], hi = w[2 * h + 1];
            const uint32_t a = (lo & 0x0F0F0F0Fu) | ((lo >> 4) & 0xF0F0F0F0u);  // bytes (b0|b1<<4) at 0, (b2|b3<<4) at 2
            const uint32_t b = (hi & 0x0F0F0F0Fu) | ((hi >> 4) & 0xF0F0F0F0u);
            o[h] = __byte_perm(a, b, 0x6420);
        }
        *reinterpret_cast<uint2 *>(out + v * 8) = make_uint2(o[0], o[1]);
    }
}

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

// Transactions [m_old, m_old + m_new) of each item (blockIdx.y strides over
// the items) from `nb` (n_in
// words per item, bit p of word j = new transaction 64 j + p) merged into the
// item's bitmap: output word o >= m_old / 64 takes the new bits shifted by
// m_old % 64, the first one keeps the old bits below that shift.  Bits of the
// input past m_new are ignored.  The popcount of the new bits is added to
// marg[item].
__global__ void append_bits_kernel(uint64_t *__restrict__ bits, int64_t wstride, int32_t n_items, int64_t m_old,
                                   const uint64_t *__restrict__ nb, int64_t n_in, int64_t m_new,
                                   unsigned long long *marg)
{
    const int64_t w0 = m_old >> 6;
    const int sh = (int)(m_old & 63);
    const int64_t n_out = ((m_old + m_new + 63) >> 6) - w0;
    const int64_t last = (m_new + 63) >> 6;  // input words that hold new bits
    for (int it = blockIdx.y; it < n_items; it += gridDim.y) {
        const uint64_t *src = nb + (int64_t)it * n_in;
        auto word = [&](int64_t j) -> uint64_t {
            if (j < 0 || j >= last) return 0ull;
            uint64_t x = src[j];
            if (j == last - 1 && (m_new & 63)) x &= (~0ull) >> (64 - (m_new & 63));
            return x;
        };
        unsigned long long c = 0;
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_out;
             j += (int64_t)gridDim.x * blockDim.x) {
            const uint64_t cur = word(j);
            c += __popcll(cur);
            uint64_t v;
            if (sh == 0) {
                v = cur;
            } else {
                v = (cur << sh) | (word(j - 1) >> (64 - sh));
                if (j == 0) v |= bits[(int64_t)it * wstride + w0] & ((1ull << sh) - 1ull);
            }
            bits[(int64_t)it * wstride + w0 + j] = v;
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(marg + it, c);
    }
}

}  // namespace

cudaError_t launch_pack_bits(const uint8_t *D, int64_t m_pad, int64_t m, int32_t n,
                             const int32_t *d_arity, const int32_t *d_soff, uint64_t *bits,
                             int64_t wstride, int32_t /*max_arity*/, int32_t *bad_state,
                             cudaStream_t s, int64_t first_word, int64_t *delta, int first_from)
{
    const int64_t words = (m + 63) / 64 - first_word;
    if (words <= 0) return cudaSuccess;
    const int64_t groups = (words + 31) / 32;  // 32 words per warp
    dim3 grid((unsigned)((groups + kPackWarps - 1) / kPackWarps), (unsigned)n);
    pack_bits_kernel<<<grid, kPackWarps * 32, 0, s>>>(D, m_pad, m, first_word, d_arity, d_soff, bits, wstride,
                                                 bad_state, reinterpret_cast<unsigned long long *>(delta),
                                                 first_from);
    return cudaGetLastError();
}

namespace {
unsigned append_grid(int64_t units, int threads)
{
    const int64_t b = (units + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 1024));
}
unsigned append_rows(int32_t n) { return (unsigned)std::max(1, std::min(n, 65535)); }
}  // namespace

cudaError_t launch_append_bits(uint64_t *bits, int64_t wstride, int32_t n_items, int64_t m_old,
                               const uint64_t *nb, int64_t n_in, int64_t m_new, int64_t *marg, cudaStream_t s)
{
    if (m_new <= 0) return cudaSuccess;
    const int64_t n_out = ((m_old + m_new + 63) >> 6) - (m_old >> 6);
    append_bits_kernel<<<dim3(append_grid(n_out, 256), append_rows(n_items)), 256, 0, s>>>(
        bits, wstride, n_items, m_old, nb, n_in, m_new, reinterpret_cast<unsigned long long *>(marg));
    return cudaGetLastError();
}

cudaError_t launch_bit_popcounts(const uint64_t *bits, int64_t rows, int64_t wstride,
                                 int64_t *counts, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    bit_popcount_kernel<<<(unsigned)rows, 256, 0, s>>>(bits, wstride, counts);
    return cudaGetLastError();
}

cudaError_t launch_pack_codes4(const uint8_t *D, int64_t m_pad, int32_t n, int64_t row0, int64_t row1,
                               uint8_t *D4, cudaStream_t s)
{
    row0 &= ~(int64_t)15;
    row1 = std::min<int64_t>(m_pad, (row1 + 15) & ~(int64_t)15);
    if (n <= 0 || row1 <= row0) return cudaSuccess;
    const int64_t vecs = (row1 - row0) / 16;
    dim3 grid((unsigned)std::min<int64_t>((vecs + 255) / 256, 65535), (unsigned)n);
    pack_codes4_kernel<<<grid, 256, 0, s>>>(D, m_pad, row0, vecs, D4);
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
