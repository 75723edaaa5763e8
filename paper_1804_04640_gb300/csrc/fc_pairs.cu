// fc_pairs.cu -- every pairwise contingency table at once on tcgen05 tensor
// cores.
//
// Let A be the m x R one-hot matrix of D (R = sum of arities, column
// soff_i + s of row p is 1 when X_i = s in instance p; its columns are the
// per-state bitmaps of Sec. 3.2).  Then C = A^T A holds, for variables a < b,
// the Sec. 2 contingency table of the pair (a, b) in its block
// (soff_a.., soff_b..), and the marginal counts on its diagonal.  This is a
// dense contraction over the m instances, so it runs on the tensor cores:
//
//   * operands are built on the fly from the bitmaps: each bit becomes one
//     e4m3 byte, 0x08 (= 2^-6, the smallest normal) or 0, written K-major into
//     shared memory with the 128-byte swizzle the MMA descriptors describe;
//   * a CTA owns a 256 x 256 region of C and one range of rows (split K):
//     two tcgen05.mma.cta_group::1.kind::f8f6f4 accumulators (M = 128,
//     N <= 256, K = 32, FP32 in tensor memory, 512 columns) share one B
//     operand; on diagonal regions both A halves are slices of B, so only B
//     is built.  Every product is 0 or 2^-12 and every partial sum is 2^-12
//     times an integer no larger than the rows of one split, which the
//     planner keeps far below 2^24, so the FP32 sums are exact; the result is
//     read with tcgen05.ld, scaled by 2^12, converted to int32 and added to C;
//   * only regions on or above the diagonal of C are computed, and in each
//     an accumulator multiplies only the columns it needs: those inside the
//     R x R matrix (rounded up to 16, the MMA's N granule), and on the
//     diagonal the second half skips the quarter below the diagonal.  Rows
//     of B past R are zero, filled once per stage buffer; the planner splits
//     each region's rows over CTAs in proportion to its shared-memory
//     traffic, so that every CTA of the one wave finishes at about the same
//     time.
//
// Pipeline per CTA: 16 producer warps fill kStages shared-memory stages
// (loading the bitmap words three stages ahead of the one they expand) and
// signal a "full" mbarrier; the MMA thread waits for it, issues eight MMAs and
// commits to the stage's "empty" mbarrier.  Every wait is bounded by
// `wait_limit` polls; a wait that runs out sets the status word and the CTA
// winds down (no trap, TMEM always released).
#include "fc_internal.h"
#include "fc_score.cuh"

namespace fc {
namespace {

constexpr int kM = 128;                      // rows of one MMA
constexpr int kN = 256;                      // columns of one MMA
constexpr int kRegion = 256;                 // a CTA's region of C is kRegion x kRegion
constexpr int kKStage = 128;                 // instances per stage = bytes per operand row
constexpr int kStages = 3;
constexpr int kProducerWarps = 16;
constexpr int kProducers = kProducerWarps * 32;
constexpr int kThreads = kProducers + 32;    // + the MMA / TMEM warp
constexpr int kABytes = kRegion * kKStage;   // two A halves of 128 rows, 32 KiB
constexpr int kBBytes = kN * kKStage;        // 32 KiB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr uint32_t kTmemCols = 512;          // two 128 x 256 FP32 accumulators

// Instruction descriptor of kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3
// (format 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_n(int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle (layout 2 at bit
// 61), 8-row core groups 1024 bytes apart (SBO), version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int64_t limit)
{
    for (int64_t i = 0; i < limit; ++i)
        if (mbar_try(a, parity)) return true;
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Four bits -> four e4m3 bytes (0x08 = 2^-6 where the bit is set).  The
// multiply places bit i at bit 8i + 3; its four shifted copies are 7 bits
// apart, so no carries occur.
__device__ __forceinline__ uint32_t expand4(uint32_t nib)
{
    return (nib * 0x01020408u) & 0x08080808u;
}

constexpr float kOneHotScale = 4096.0f;  // 1 / (2^-6 * 2^-6)

__device__ __forceinline__ void store_row_word(uint8_t *tile, int row, int half, uint64_t w)
{
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const uint32_t x = (uint32_t)(w >> (16 * cc)) & 0xFFFFu;
        uint4 v;
        v.x = expand4(x & 0xFu);
        v.y = expand4((x >> 4) & 0xFu);
        v.z = expand4((x >> 8) & 0xFu);
        v.w = expand4((x >> 12) & 0xFu);
        const int chunk = 4 * half + cc;
        *reinterpret_cast<uint4 *>(tile + row * 128 + ((chunk ^ (row & 7)) << 4)) = v;
    }
}

__global__ void __launch_bounds__(kThreads, 1) pairs_gemm_kernel(const PairsParams P)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + kStages * kStageBytes);  // full[S], empty[S], acc
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's region: the last one whose first CTA is at or before it
    int lo = 0, hi = P.nregions - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.regions[mid].cta0 <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const PairsRegion G = P.regions[lo];
    const int split = (int)blockIdx.x - G.cta0;
    const bool diag = G.ra == G.rb;  // both A halves are slices of B
    const int64_t total_stages = (P.words + 1) / 2;
    const int64_t st0 = total_stages * split / G.ksplit;
    const int64_t st1 = total_stages * (split + 1) / G.ksplit;
    const int64_t nst = st1 - st0;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), accb = smem_u32(bars + 2 * kStages);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, kProducers);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kProducerWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < kProducerWarps) {
        // ---------------------------------------------------------- producers
        // B rows past the matrix that the MMAs read (up to N's 16-row granule,
        // and on the diagonal the rows the A halves take from B) are zero in
        // every stage buffer, written once
        const int bread = diag ? max((G.real_b + 15) & ~15, G.n1 > 0 ? kRegion : kM) : (G.real_b + 15) & ~15;
        for (int u = threadIdx.x; u < kStages * (bread - G.real_b) * 8; u += kProducers) {
            const int slot = u / ((bread - G.real_b) * 8), r = u % ((bread - G.real_b) * 8);
            uint8_t *b_tile = smem + slot * kStageBytes + kABytes;
            *reinterpret_cast<uint4 *>(b_tile + (G.real_b + (r >> 3)) * 128 + ((r & 7) << 4)) = make_uint4(0, 0, 0, 0);
        }
        // tasks: (operand row, half of the stage's two 64-bit words); off the
        // diagonal rows 0..255 are the A halves and 256.. are B, on it all
        // rows are B
        constexpr int kTasksMax = ((kRegion + kN) * 2 + kProducers - 1) / kProducers;
        const int a_rows = diag ? 0 : kRegion;
        const int ntask = (a_rows + G.real_b) * 2;
        // The words of three stages are in flight: the loop is unrolled by
        // three so that each buffer keeps its registers (a register copy of a
        // pending load would wait for it) and is refilled, three stages
        // ahead, right after its stage has been expanded.
        uint64_t q0[kTasksMax], q1[kTasksMax], q2[kTasksMax];
        auto load = [&](int64_t st, uint64_t (&dst)[kTasksMax]) {
            const int64_t kw = (st0 + st) * 2;  // first 64-bit word of that stage
#pragma unroll
            for (int j = 0; j < kTasksMax; ++j) {
                const int u = threadIdx.x + j * kProducers;
                const int i = u >> 1, half = u & 1;
                const int grow = i < a_rows ? G.ra * kRegion + i : G.rb * kRegion + (i - a_rows);
                dst[j] = (st < nst && u < ntask && grow < P.R)
                             ? __ldg(P.bits + (int64_t)grow * P.wstride + kw + half)
                             : 0ull;
            }
        };
        // expands stage st from cur into its slot; false when the CTA aborts
        auto stage = [&](int64_t st, const uint64_t (&cur)[kTasksMax]) -> bool {
            const int slot = (int)(st % kStages);
            if (st >= kStages) {
                if (!mbar_wait(empty0 + 8 * slot, (uint32_t)((st / kStages - 1) & 1), P.wait_limit)) {
                    atomicExch(&s_abort, 1);
                    return false;
                }
            }
            if (*(volatile int *)&s_abort) return false;
            uint8_t *a_tile = smem + slot * kStageBytes;
            uint8_t *b_tile = a_tile + kABytes;
#pragma unroll
            for (int j = 0; j < kTasksMax; ++j) {
                const int u = threadIdx.x + j * kProducers;
                if (u < ntask) {
                    const int i = u >> 1, half = u & 1;
                    if (i < a_rows)
                        store_row_word(a_tile, i, half, cur[j]);
                    else
                        store_row_word(b_tile, i - a_rows, half, cur[j]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(full0 + 8 * slot);
            return true;
        };
        load(0, q0);
        load(1, q1);
        load(2, q2);
        for (int64_t st = 0; st < nst; st += 3) {
            if (!stage(st, q0)) break;
            load(st + 3, q0);
            if (st + 1 >= nst || !stage(st + 1, q1)) break;
            load(st + 4, q1);
            if (st + 2 >= nst || !stage(st + 2, q2)) break;
            load(st + 5, q2);
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issuer
        const uint32_t id0 = G.n0 > 0 ? idesc_n(G.n0) : 0u, id1 = G.n1 > 0 ? idesc_n(G.n1) : 0u;
        for (int64_t st = 0; st < nst; ++st) {
            const int slot = (int)(st % kStages);
            if (!mbar_wait(full0 + 8 * slot, (uint32_t)((st / kStages) & 1), P.wait_limit) ||
                *(volatile int *)&s_abort) {
                atomicExch(&s_abort, 1);
                break;
            }
            tc_fence_after();
            const uint32_t b_addr = smem_u32(smem + slot * kStageBytes) + kABytes;
            const uint32_t a_addr = diag ? b_addr : b_addr - kABytes;
            const uint32_t b1_addr = b_addr + (uint32_t)G.coff1 * kKStage;  // B rows from coff1 on
#pragma unroll
            for (int kk = 0; kk < kKStage / 32; ++kk) {
                const uint32_t acc = (st > 0 || kk > 0) ? 1u : 0u;
                if (G.n0 > 0)  // rows 0..127
                    mma_f8(tmem, smem_desc(a_addr + 32 * kk), smem_desc(b_addr + 32 * kk), id0, acc);
                if (G.n1 > 0)  // rows 128..255
                    mma_f8(tmem + kN, smem_desc(a_addr + kM * kKStage + 32 * kk), smem_desc(b1_addr + 32 * kk), id1,
                           acc);
            }
            mma_commit(empty0 + 8 * slot);
        }
        mma_commit(accb);  // fires when every MMA issued above has completed
    }

    // -------------------------------------------------------------- epilogue
    if (warp < 4 && nst > 0) {
        const bool done = mbar_wait(accb, 0u, P.wait_limit);
        if (!done) atomicExch(&s_abort, 1);
        tc_fence_after();
        // warp-uniform decision: tcgen05.ld below is a warp-wide instruction
        if (__all_sync(kFull, done && !*(volatile int *)&s_abort)) {
#pragma unroll 1
          for (int half = 0; half < 2; ++half) {
            const int n = half ? G.n1 : G.n0;
            const int coff = half ? G.coff1 : 0;
            const int row = G.ra * kRegion + half * kM + warp * 32 + lane;
            int32_t *crow = P.C + (int64_t)row * P.R_pad + G.rb * kRegion + coff;
#pragma unroll 1
            for (int c0 = 0; c0 < n; c0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(half * kN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                      "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                      "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < P.R) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        // columns of the accumulator only; the lower triangle is never read
                        const int col = G.rb * kRegion + coff + c0 + j;
                        const int v = __float2int_rn(__uint_as_float(r[j]) * kOneHotScale);
                        if (c0 + j < n && v && col < P.R && row <= col) atomicAdd(crow + c0 + j, v);
                    }
                }
            }
          }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_abort) atomicExch(P.status, kStatusTimeout);
    if (warp == kProducerWarps) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

// Pair tables and their mutual information, one warp per pair (a, b), a < b.
__global__ void pairs_extract_kernel(const int32_t *__restrict__ C, int32_t R_pad, int32_t n,
                                     const int32_t *__restrict__ arity, const int32_t *__restrict__ soff,
                                     const int64_t *__restrict__ pair_off, int64_t m, int32_t *tables,
                                     float *mi)
{
    const int a = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int ra = arity[a], sa = soff[a];
    const int64_t base = (int64_t)a * n - (int64_t)a * (a + 1) / 2;  // pairs (a', b) with a' < a
    for (int b = a + 1 + warp; b < n; b += nwarps) {
        const int rb = arity[b], sb = soff[b];
        const int64_t pidx = base + (b - a - 1);
        Kahan acc{0.0f, 0.0f};
        for (int cell = lane; cell < ra * rb; cell += 32) {
            const int x = cell / rb, y = cell % rb;
            const int32_t nxy = C[(int64_t)(sa + x) * R_pad + sb + y];
            if (tables) tables[pair_off[pidx] + cell] = nxy;
            if (mi) {
                const int64_t nx = C[(int64_t)(sa + x) * R_pad + sa + x];
                const int64_t ny = C[(int64_t)(sb + y) * R_pad + sb + y];
                if (nx > 0 && ny > 0) {
                    const long long num = (long long)nxy * m - (long long)nx * ny;
                    const float xr = (float)num / ((float)nx * (float)ny);
                    kahan_add(acc, ((float)nx / (float)m) * ((float)ny / (float)m) * mi_term(xr));
                }
            }
        }
        if (mi) {
            for (int o = 16; o > 0; o >>= 1) {
                Kahan other{__shfl_xor_sync(kFull, acc.s, o), __shfl_xor_sync(kFull, acc.c, o)};
                kahan_merge(acc, other);
            }
            if (lane == 0) mi[pidx] = __fsub_rn(acc.s, acc.c) * kInvLn2;
        }
    }
}

// A wait on an mbarrier nothing arrives at: exercises the bounded-wait path.
__global__ void wait_selftest_kernel(int32_t *status, int64_t limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(smem_u32(&bar), 0u, limit)) atomicExch(status, kStatusTimeout);
    }
}

}  // namespace

cudaError_t launch_pairs_gemm(const PairsParams &p, cudaStream_t s)
{
    if (p.R_pad % kRegion != 0 || p.nregions < 1 || p.grid < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(pairs_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    pairs_gemm_kernel<<<p.grid, kThreads, kSmemBytes, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_pairs_extract(const int32_t *C, int32_t R_pad, int32_t n, const int32_t *d_arity,
                                 const int32_t *d_soff, const int64_t *d_pair_off, int64_t m,
                                 int32_t *pair_tables, float *mi, cudaStream_t s)
{
    if (n < 2) return cudaSuccess;
    pairs_extract_kernel<<<n - 1, 256, 0, s>>>(C, R_pad, n, d_arity, d_soff, d_pair_off, m, pair_tables, mi);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int32_t *status, int64_t wait_limit, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(status, wait_limit);
    return cudaGetLastError();
}

}  // namespace fc
