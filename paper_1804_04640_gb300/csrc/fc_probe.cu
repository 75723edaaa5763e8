// fc_probe.cu -- throughput probes of the on-chip units the counting kernels
// are bound by, the denominators of their rooflines.
//
// The histogram strategy (keys counted in shared memory) reads its columns
// from L2 and issues one shared-memory atomic per instance; the itemset and
// all-splits kernels issue a 64-bit AND, a population count and an add per
// word of every (sub)set.  HBM bandwidth bounds none of them on the workloads
// whose database fits in L2, so each probe measures one of these rates on its
// own, with every lane busy and nothing else in the loop:
//   L2 read       16-byte loads that bypass L1 (ld.global.cg) over a buffer
//                 that stays in L2, GB/s;
//   shared atomic conflict-free atomicAdd(+1) to shared memory (every lane
//                 of a warp on its own bank), atomics/s;
//   AND+popcount  c += popcount(a & b) on 64-bit register words, words/s.
#include "fc_host.h"

namespace fc {
namespace {

// Virtual index v = 0 .. total - 1 reads 16-byte word v mod n16 (n16 a power
// of two): consecutive lanes read consecutive words, and since the grid's
// stride is not a multiple of n16 each pass over the buffer reaches an SM
// through different lines than the pass before.
__global__ void __launch_bounds__(512) probe_l2_read(const uint4 *__restrict__ buf, uint32_t mask, uint32_t total,
                                                     uint32_t *sink)
{
    uint32_t acc = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
#pragma unroll 4
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < total; v += stride) {
        const uint4 x = __ldcg(buf + (v & mask));
        acc ^= x.x ^ x.y ^ x.z ^ x.w;
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads alive
}

constexpr int kAtomicWords = 64 * 32;

__global__ void __launch_bounds__(256) probe_smem_atomic(int iters, int32_t *sink)
{
    __shared__ int32_t tab[kAtomicWords];
    for (int i = threadIdx.x; i < kAtomicWords; i += blockDim.x) tab[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int row = (threadIdx.x >> 5) * 5;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) atomicAdd(&tab[((row + u) & 63) * 32 + lane], 1);
        row += 17;
    }
    __syncthreads();
    if (tab[threadIdx.x] == -1) sink[0] = 1;
}

__global__ void __launch_bounds__(256) probe_and_popc(int iters, uint64_t seed, unsigned long long *sink)
{
    uint64_t a[8];
    const uint64_t t = seed ^ ((uint64_t)(blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B97F4A7C15ull);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = t * (2 * j + 1) + (t >> (j + 7));
    uint64_t b = t | 1u;
    uint32_t c = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) c += (uint32_t)__popcll(a[j] & b);
        b = (b << 1) | (b >> 63);  // next word: a rotation, so no AND can be hoisted
    }
    if (c == 0xFFFFFFFFu) sink[0] = c;
}

}  // namespace
}  // namespace fc

extern "C" int fc_probe_rate(int32_t kind, int64_t size, double *rate, void *stream)
{
    using namespace fc;
    if (!rate) return fail(FC_ERR_ARG, "fc_probe_rate: null rate");
    if (kind < FC_PROBE_L2_READ || kind > FC_PROBE_AND_POPC) return fail(FC_ERR_ARG, "fc_probe_rate: unknown kind %d", kind);
    if (kind == FC_PROBE_L2_READ && (size < (1 << 20) || size > ((int64_t)64 << 20) || (size & (size - 1))))
        return fail(FC_ERR_ARG, "fc_probe_rate: the L2 buffer must be a power of two from 1 MiB to 64 MiB");
    int dev = 0, sms = 0;
    FC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    cudaStream_t s = (cudaStream_t)stream;
    void *buf = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FC_OK;
    double units = 0.0, best_ms = 0.0;
    // one full wave: every SM holds as many CTAs as fit
    int occ_l2 = 1, occ_at = 1, occ_pc = 1;
    FC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_l2, probe_l2_read, 512, 0), "occupancy");
    FC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_at, probe_smem_atomic, 256, 0), "occupancy");
    FC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_pc, probe_and_popc, 256, 0), "occupancy");
    auto run = [&](int what) -> cudaError_t {
        switch (kind) {
        case FC_PROBE_L2_READ: {
            // about 2 GiB per timed launch
            const int64_t reps = what ? std::max<int64_t>(32, ((int64_t)2 << 30) / size) : 1;
            const uint32_t n16 = (uint32_t)(size / 16);
            probe_l2_read<<<sms * occ_l2, 512, 0, s>>>((const uint4 *)buf, n16 - 1, (uint32_t)(n16 * reps),
                                                  (uint32_t *)sink);
            units = (double)size * reps;
            break;
        }
        case FC_PROBE_SMEM_ATOMIC: {
            const int iters = what ? 4096 : 16;
            probe_smem_atomic<<<sms * occ_at, 256, 0, s>>>(iters, (int32_t *)sink);
            units = (double)sms * occ_at * 256 * iters * 16;
            break;
        }
        default: {
            const int iters = what ? 8192 : 16;
            probe_and_popc<<<sms * occ_pc, 256, 0, s>>>(iters, 0x2545F4914F6CDD1Dull, (unsigned long long *)sink);
            units = (double)sms * occ_pc * 256 * iters * 8;
            break;
        }
        }
        return cudaGetLastError();
    };
    cudaError_t e;
    if ((e = cudaMalloc(&sink, 64)) != cudaSuccess) return cuda_fail(e, "cudaMalloc probe sink");
    if (kind == FC_PROBE_L2_READ) {
        if ((e = cudaMalloc(&buf, (size_t)size)) != cudaSuccess) {
            cudaFree(sink);
            return cuda_fail(e, "cudaMalloc probe buffer");
        }
        e = cudaMemsetAsync(buf, 0x5A, (size_t)size, s);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one short launch brings the buffer into L2, then the best of five timed launches
    if (e == cudaSuccess) e = run(0);
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        if ((e = run(1)) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if (i == 0 || ms < best_ms) best_ms = ms;
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "fc_probe_rate");
    else *rate = units / (best_ms * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    return rc;
}
