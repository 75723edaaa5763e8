// fc_ctx.cu -- contexts behind the C ABI: error state, loading a database or
// transaction bitmaps (column-major D, per-state bitmaps, marginals,
// entropies), growing it by appends (Sec. 6), freeing it, the host worker
// threads and the pinned descriptor staging.
#include "fc_host.h"

#include <cmath>
#include <cstdio>

using namespace fc;

// ------------------------------------------------------------------ errors

namespace fc {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int set_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(FC_ERR_OOM, "%s: out of device memory", what);
    }
    return fail(FC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Pinned host staging of at least `bytes` for plan descriptors, free of any
// copy still reading it; nullptr on failure.
uint8_t *stage_host(fc_ctx *c, size_t bytes)
{
    fc_ctx::Stage &st = c->stage[c->bank];
    if (st.ev && cudaEventSynchronize(st.ev) != cudaSuccess) return nullptr;
    if (bytes > st.bytes) {
        const size_t want = std::max(bytes, st.bytes + st.bytes / 2);
        if (st.h) cudaFreeHost(st.h);
        st.h = nullptr;
        st.bytes = 0;
        if (cudaHostAlloc((void **)&st.h, want, cudaHostAllocDefault) != cudaSuccess) {
            st.h = nullptr;
            return nullptr;
        }
        st.bytes = want;
    }
    if (!st.ev && cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return st.h;
}
uint8_t *stage_grow(fc_ctx *c, size_t bytes, size_t keep)
{
    fc_ctx::Stage &st = c->stage[c->bank];
    if (bytes <= st.bytes) return st.h;
    if (st.ev && cudaEventSynchronize(st.ev) != cudaSuccess) return nullptr;
    const size_t want = std::max(bytes, st.bytes + st.bytes / 2);
    uint8_t *h = nullptr;
    if (cudaHostAlloc((void **)&h, want, cudaHostAllocDefault) != cudaSuccess) return nullptr;
    if (st.h) {
        std::memcpy(h, st.h, std::min(keep, st.bytes));
        cudaFreeHost(st.h);
    }
    st.h = h;
    st.bytes = want;
    return h;
}
cudaError_t upload_stage(fc_ctx *c, void *dst, size_t bytes)
{
    fc_ctx::Stage &st = c->stage[c->bank];
    cudaError_t e = cudaMemcpyAsync(dst, st.h, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(st.ev, c->stream);
    return e;
}

}  // namespace fc

extern "C" const char *fc_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------- host worker threads

int fc::host_threads(fc_ctx *c)
{
    if (!c->pool_threads) {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        c->pool_threads.reset(new (std::nothrow) PlanPool());
        if (c->pool_threads) c->pool_threads->start(std::max(0, std::min(7, hw - 1)));
    }
    return c->pool_threads ? c->pool_threads->size() : 1;
}

void fc::run_host_threads(fc_ctx *c, int n, const std::function<void(int)> &f)
{
    if (n <= 1 || !c->pool_threads) {
        for (int i = 0; i < std::max(n, 0); ++i) f(i);
        return;
    }
    c->pool_threads->run(std::min(n, c->pool_threads->size()), f);
}


// ---------------------------------------------------------------- loading

namespace {

int finish_load(fc_ctx *c)
{
    // marginal counts per (variable, state) and entropies (DFS order, Sec. 3.2)
    FC_CUDA(cudaMalloc(&c->d_marg, sizeof(int64_t) * std::max(c->R, 1)), "cudaMalloc marginals");
    FC_CUDA(launch_bit_popcounts(c->d_bits, c->R, c->wstride, c->d_marg, c->stream), "popcounts");
    c->marg.assign(c->R, 0);
    FC_CUDA(cudaMemcpyAsync(c->marg.data(), c->d_marg, sizeof(int64_t) * c->R,
                            cudaMemcpyDeviceToHost, c->stream), "copy marginals");
    FC_CUDA(cudaStreamSynchronize(c->stream), "load");
    c->entropy.assign(c->n, 0.0);
    if (!c->transactions) {
        for (int i = 0; i < c->n; ++i) {
            double h = 0.0;
            for (int s = 0; s < c->arity[i]; ++s) {
                const double p = (double)c->marg[c->soff[i] + s] / (double)c->m;
                if (p > 0.0) h -= p * std::log2(p);
            }
            c->entropy[i] = h;
        }
    }
    c->mark.assign(c->n, 0u);
    c->entropy_stale = true;
    return FC_OK;
}

int new_ctx(fc_ctx **out, int32_t n, int64_t m)
{
    fc_ctx *c = new (std::nothrow) fc_ctx();
    if (!c) return fail(FC_ERR_OOM, "host allocation failed");
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    c->n = n;
    c->m = m;
    c->words = (m + 63) / 64;
    c->wstride = round_up(c->words, kChunkWords);
    *out = c;
    e = cudaMalloc(&c->d_status, 16);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 16, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    return FC_OK;
}

}  // namespace

namespace {
// The 4-bit copy of D (fc_ctx::d_D4) for a database whose arities are all at
// most 16, allocated for the current m_pad and packed for rows [0, m).
cudaError_t build_codes4(fc_ctx *c)
{
    if (c->transactions || c->n > 65535) return cudaSuccess;
    for (const int32_t r : c->arity)
        if (r > 16) return cudaSuccess;
    const size_t bytes = (size_t)c->n * (size_t)(c->m_pad / 2);
    cudaError_t e = cudaMalloc(&c->d_D4, bytes);
    if (e == cudaErrorMemoryAllocation) {  // optional: the byte columns serve every query
        (void)cudaGetLastError();
        c->d_D4 = nullptr;
        return cudaSuccess;
    }
    if (e != cudaSuccess) {
        c->d_D4 = nullptr;
        return e;
    }
    e = cudaMemsetAsync(c->d_D4, 0, bytes, c->stream);
    if (e == cudaSuccess) e = launch_pack_codes4(c->d_D, c->m_pad, c->n, 0, c->m, c->d_D4, c->stream);
    return e;
}
}  // namespace

extern "C" int fc_load(fc_ctx **out, const uint8_t *D, int32_t n, int64_t m,
                       const int32_t *arities, int32_t layout, int32_t where)
{
    if (!out || !D || !arities) return fail(FC_ERR_ARG, "fc_load: null argument");
    *out = nullptr;
    if (n < 1 || m < 1) return fail(FC_ERR_ARG, "fc_load: need n >= 1 and m >= 1");
    if (m >= ((int64_t)1 << 31)) return fail(FC_ERR_RANGE, "fc_load: m must be < 2^31");
    if (layout != FC_COL_MAJOR && layout != FC_ROW_MAJOR) return fail(FC_ERR_ARG, "fc_load: bad layout");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_load: bad pointer location");
    for (int i = 0; i < n; ++i)
        if (arities[i] < 1 || arities[i] > 255)
            return fail(FC_ERR_ARG, "fc_load: arity of variable %d is %d, not in 1..255", i, arities[i]);
    fc_ctx *c = nullptr;
    int rc = new_ctx(&c, n, m);
    if (rc != FC_OK) {
        fc_free(c);
        return rc;
    }
    c->arity.assign(arities, arities + n);
    c->soff.resize(n);
    for (int i = 0; i < n; ++i) {
        c->soff[i] = c->R;
        c->R += arities[i];
    }
    c->m_pad = round_up(m, kChunkRows);
    auto bail = [&](int code) {
        fc_free(c);
        return code;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_D, (size_t)n * c->m_pad)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc D"));
    if ((e = cudaMemsetAsync(c->d_D, 0, (size_t)n * c->m_pad, c->stream)) != cudaSuccess) return bail(cuda_fail(e, "memset D"));
    const cudaMemcpyKind kind = where == FC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (layout == FC_COL_MAJOR) {
        e = cudaMemcpy2DAsync(c->d_D, c->m_pad, D, m, m, n, kind, c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(e, "copy D"));
    } else {
        uint8_t *tmp = nullptr;
        if ((e = cudaMalloc(&tmp, (size_t)n * m)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc D rows"));
        e = cudaMemcpyAsync(tmp, D, (size_t)n * m, kind, c->stream);
        if (e == cudaSuccess) e = launch_transpose_rows(tmp, m, n, c->d_D, c->m_pad, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return bail(cuda_fail(e, "transpose D"));
    }
    if ((e = cudaMalloc(&c->d_arity, sizeof(int32_t) * n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&c->d_soff, sizeof(int32_t) * n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    cudaMemcpyAsync(c->d_arity, c->arity.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_soff, c->soff.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream);
    // one row per (variable, state) plus an all-zero row R (states outside an arity)
    const size_t bits_bytes = sizeof(uint64_t) * (size_t)(c->R + 1) * c->wstride;
    if ((e = cudaMalloc(&c->d_bits, bits_bytes)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc bitmaps"));
    if ((e = cudaMemsetAsync(c->d_bits, 0, bits_bytes, c->stream)) != cudaSuccess) return bail(cuda_fail(e, "memset bitmaps"));
    int32_t *bad = c->d_status + 1;
    e = launch_pack_bits(c->d_D, c->m_pad, m, n, c->d_arity, c->d_soff, c->d_bits, c->wstride, 255, bad, c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pack bitmaps"));
    int32_t bad_h = 0;
    e = cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "load"));
    if (bad_h) return bail(fail(FC_ERR_RANGE, "fc_load: a stored state is >= its variable's arity"));
    cudaMemsetAsync(c->d_status, 0, 16, c->stream);
    if ((e = build_codes4(c)) != cudaSuccess) return bail(cuda_fail(e, "4-bit codes"));
    rc = finish_load(c);
    if (rc != FC_OK) return bail(rc);
    *out = c;
    return FC_OK;
}

extern "C" int fc_load_bits(fc_ctx **out, const uint64_t *bitmaps, int32_t n_items, int64_t m,
                            int32_t where)
{
    if (!out || !bitmaps) return fail(FC_ERR_ARG, "fc_load_bits: null argument");
    *out = nullptr;
    if (n_items < 1 || m < 1) return fail(FC_ERR_ARG, "fc_load_bits: need n_items >= 1 and m >= 1");
    if (m >= ((int64_t)1 << 31)) return fail(FC_ERR_RANGE, "fc_load_bits: m must be < 2^31");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_load_bits: bad pointer location");
    fc_ctx *c = nullptr;
    int rc = new_ctx(&c, n_items, m);
    if (rc != FC_OK) {
        fc_free(c);
        return rc;
    }
    c->transactions = true;
    c->arity.assign(n_items, 1);
    c->soff.resize(n_items);
    for (int i = 0; i < n_items; ++i) c->soff[i] = i;
    c->R = n_items;
    const size_t bits_bytes = sizeof(uint64_t) * (size_t)n_items * c->wstride;
    cudaError_t e = cudaMalloc(&c->d_bits, bits_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bits, 0, bits_bytes, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(c->d_bits, sizeof(uint64_t) * c->wstride, bitmaps, sizeof(uint64_t) * c->words,
                              sizeof(uint64_t) * c->words, n_items,
                              where == FC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = launch_mask_tail_bits(c->d_bits, n_items, c->wstride, m, c->stream);
    if (e != cudaSuccess) {
        fc_free(c);
        return cuda_fail(e, "fc_load_bits");
    }
    rc = finish_load(c);
    if (rc != FC_OK) {
        fc_free(c);
        return rc;
    }
    *out = c;
    return FC_OK;
}

extern "C" void fc_free(fc_ctx *c)
{
    if (!c) return;
    DevGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->out_stream) cudaStreamSynchronize(c->out_stream);
    // plans still alive keep their host struct for fc_plan_free but lose
    // their device memory and their context
    for (fc_plan *p : c->live_plans) {
        release_plan(p);
        p->ctx = nullptr;
    }
    c->live_plans.clear();
    for (auto &st : c->stage) {
        if (st.h) cudaFreeHost(st.h);
        if (st.ev) cudaEventDestroy(st.ev);
    }
    if (c->out_stream) cudaStreamDestroy(c->out_stream);
    for (cudaEvent_t ev : c->part_done)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->copy_done)
        if (ev) cudaEventDestroy(ev);
    for (auto &b : c->io) b.release();
    c->marg_delta.release();
    c->dplan_buf.release();
    for (auto &b : c->pipe_io) b.release();
    for (auto &bank : c->pool)
        for (auto &b : bank) b.release();
    cudaFree(c->d_D);
    cudaFree(c->d_D4);
    cudaFree(c->d_bits);
    cudaFree(c->d_marg);
    cudaFree(c->d_entropy_f);
    cudaFree(c->d_arity);
    cudaFree(c->d_soff);
    cudaFree(c->d_status);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ---------------------------------------------------------------- appends
//
// Sec. 6: a database that grows by new instances needs only an update of the
// bitmaps (and the histogram/radix strategies read D as it stands).  Storage
// keeps spare rows: D columns are m_pad bytes apart and bitmap rows wstride
// words apart, both sized for a capacity that grows geometrically, with every
// byte and bit past m zero.

namespace {

int64_t capacity_rows(const fc_ctx *c)
{
    const int64_t bit_rows = c->wstride * 64;
    return c->transactions ? bit_rows : std::min(c->m_pad, bit_rows);
}

// Make room for m_need instances (reallocating and copying when needed).
int grow_storage(fc_ctx *c, int64_t m_need)
{
    if (m_need <= capacity_rows(c)) return FC_OK;
    if (m_need >= ((int64_t)1 << 31)) return fail(FC_ERR_RANGE, "m would reach %lld, must stay < 2^31", (long long)m_need);
    int64_t cap = std::max<int64_t>(m_need, capacity_rows(c) + capacity_rows(c) / 2);
    cap = std::min<int64_t>(round_up(cap, kChunkRows), ((int64_t)1 << 31) - 1);
    cap = std::max(cap, m_need);
    const int64_t new_pad = round_up(cap, kChunkRows);
    const int64_t new_wstride = round_up((new_pad + 63) / 64, kChunkWords);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "append");
    const int64_t rows = c->transactions ? c->R : c->R + 1;
    uint64_t *nb = nullptr;
    const size_t bbytes = sizeof(uint64_t) * (size_t)rows * new_wstride;
    if ((e = cudaMalloc(&nb, bbytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc bitmaps");
    e = cudaMemsetAsync(nb, 0, bbytes, c->stream);
    if (e == cudaSuccess && c->words > 0)
        e = cudaMemcpy2DAsync(nb, sizeof(uint64_t) * new_wstride, c->d_bits, sizeof(uint64_t) * c->wstride,
                              sizeof(uint64_t) * c->words, rows, cudaMemcpyDeviceToDevice, c->stream);
    uint8_t *nd = nullptr, *nd4 = nullptr;
    if (e == cudaSuccess && !c->transactions) {
        const size_t dbytes = (size_t)c->n * new_pad;
        e = cudaMalloc(&nd, dbytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(nd, 0, dbytes, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(nd, new_pad, c->d_D, c->m_pad, c->m, c->n, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess && c->d_D4) {
            e = cudaMalloc(&nd4, dbytes / 2);
            if (e == cudaErrorMemoryAllocation) {  // drop the optional 4-bit copy instead
                (void)cudaGetLastError();
                nd4 = nullptr;
                e = cudaSuccess;
            } else if (e == cudaSuccess) {
                e = cudaMemsetAsync(nd4, 0, dbytes / 2, c->stream);
            }
            if (e == cudaSuccess && nd4)
                e = cudaMemcpy2DAsync(nd4, new_pad / 2, c->d_D4, c->m_pad / 2, (c->m + 1) / 2, c->n,
                                      cudaMemcpyDeviceToDevice, c->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(nb);
        cudaFree(nd);
        cudaFree(nd4);
        return cuda_fail(e, "grow storage");
    }
    cudaFree(c->d_bits);
    c->d_bits = nb;
    c->wstride = new_wstride;
    if (!c->transactions) {
        cudaFree(c->d_D);
        c->d_D = nd;
        if (c->d_D4) {
            cudaFree(c->d_D4);
            c->d_D4 = nd4;
        }
        c->m_pad = new_pad;
    }
    return FC_OK;
}

// New instance count, generation and entropies after an append; the host
// copy of the marginals is read back from the device unless the caller has
// already brought it up to date.
int finish_append(fc_ctx *c, int64_t m_total, bool read_marginals = true)
{
    c->m = m_total;
    c->words = (m_total + 63) / 64;
    c->generation += 1;
    if (read_marginals) {
        cudaError_t e = cudaMemcpyAsync(c->marg.data(), c->d_marg, sizeof(int64_t) * c->R,
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "append marginals");
    }
    if (!c->transactions)
        for (int i = 0; i < c->n; ++i) {
            double h = 0.0;
            for (int s = 0; s < c->arity[i]; ++s) {
                const double p = (double)c->marg[c->soff[i] + s] / (double)c->m;
                if (p > 0.0) h -= p * std::log2(p);
            }
            c->entropy[i] = h;
        }
    c->entropy_stale = true;
    return FC_OK;
}

}  // namespace

extern "C" int fc_reserve(fc_ctx *c, int64_t m_total)
{
    if (!c) return fail(FC_ERR_ARG, "fc_reserve: null context");
    if (m_total < 0) return fail(FC_ERR_ARG, "fc_reserve: m_total < 0");
    DevGuard g(c->device);
    return grow_storage(c, m_total);
}

extern "C" int fc_append(fc_ctx *c, const uint8_t *D, int64_t m_new, int32_t layout, int32_t where)
{
    if (!c) return fail(FC_ERR_ARG, "fc_append: null context");
    if (c->transactions) return fail(FC_ERR_STATE, "fc_append: a context from fc_load_bits takes fc_append_bits");
    if (m_new < 0) return fail(FC_ERR_ARG, "fc_append: m_new < 0");
    if (m_new == 0) return FC_OK;
    if (!D) return fail(FC_ERR_ARG, "fc_append: null D");
    if (layout != FC_COL_MAJOR && layout != FC_ROW_MAJOR) return fail(FC_ERR_ARG, "fc_append: bad layout");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_append: bad pointer location");
    DevGuard g(c->device);
    const int64_t m0 = c->m, m1 = m0 + m_new;
    int rc = grow_storage(c, m1);
    if (rc != FC_OK) return rc;
    const cudaMemcpyKind kind = where == FC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e;
    if (layout == FC_COL_MAJOR) {
        e = cudaMemcpy2DAsync(c->d_D + m0, c->m_pad, D, m_new, m_new, c->n, kind, c->stream);
    } else {
        const size_t bytes = (size_t)c->n * m_new;
        e = c->io[2].ensure(bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->io[2].p, D, bytes, kind, c->stream);
        if (e == cudaSuccess)
            e = launch_transpose_rows((const uint8_t *)c->io[2].p, m_new, c->n, c->d_D + m0, c->m_pad, c->stream);
    }
    // The repack of the bitmap words from m0 / 64 on also checks the states
    // and counts the new instances per state.  A bad state appends nothing:
    // the new rows of D are zeroed and the same words repacked over the old
    // rows alone, before m or the marginals move.
    int32_t *bad = c->d_status + 1;
    int32_t bad_h = 0;
    c->h_marg_delta.assign(c->R, 0);
    if (e == cudaSuccess) e = c->marg_delta.ensure(sizeof(int64_t) * c->R);
    int64_t *delta = (int64_t *)c->marg_delta.p;
    if (e == cudaSuccess) e = cudaMemsetAsync(delta, 0, sizeof(int64_t) * c->R, c->stream);
    if (e == cudaSuccess)
        e = launch_pack_bits(c->d_D, c->m_pad, m1, c->n, c->d_arity, c->d_soff, c->d_bits, c->wstride, 255, bad,
                             c->stream, m0 / 64, delta, (int)(m0 % 64));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->h_marg_delta.data(), delta, sizeof(int64_t) * c->R, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fc_append");
    if (bad_h) {
        // D past m0 back to zero; the partial word at m0 / 64 repacked from
        // the old rows alone; the words after it cleared in every bitmap row
        const int64_t w_old = (m0 + 63) / 64, w_new = (m1 + 63) / 64;
        cudaMemset2DAsync(c->d_D + m0, c->m_pad, 0, m_new, c->n, c->stream);
        if (m0 % 64) launch_pack_bits(c->d_D, c->m_pad, m0, c->n, c->d_arity, c->d_soff, c->d_bits, c->wstride,
                                      255, bad, c->stream, m0 / 64);
        if (w_new > w_old)
            cudaMemset2DAsync(c->d_bits + w_old, sizeof(uint64_t) * c->wstride, 0, sizeof(uint64_t) * (w_new - w_old),
                              c->R, c->stream);
        cudaMemsetAsync(bad, 0, sizeof(int32_t), c->stream);
        cudaStreamSynchronize(c->stream);
        return fail(FC_ERR_RANGE, "fc_append: a state is >= its variable's arity; nothing was appended");
    }
    for (int r = 0; r < c->R; ++r) c->marg[r] += c->h_marg_delta[r];
    e = cudaMemcpyAsync(c->d_marg, c->marg.data(), sizeof(int64_t) * c->R, cudaMemcpyHostToDevice, c->stream);
    // the 4-bit codes of the appended rows (from the 16-row group holding m0)
    if (e == cudaSuccess && c->d_D4) e = launch_pack_codes4(c->d_D, c->m_pad, c->n, m0, m1, c->d_D4, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fc_append marginals");
    return finish_append(c, m1, false);
}

extern "C" int fc_append_bits(fc_ctx *c, const uint64_t *bitmaps, int64_t m_new, int32_t where)
{
    if (!c) return fail(FC_ERR_ARG, "fc_append_bits: null context");
    if (!c->transactions) return fail(FC_ERR_STATE, "fc_append_bits: a categorical context takes fc_append");
    if (m_new < 0) return fail(FC_ERR_ARG, "fc_append_bits: m_new < 0");
    if (m_new == 0) return FC_OK;
    if (!bitmaps) return fail(FC_ERR_ARG, "fc_append_bits: null bitmaps");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_append_bits: bad pointer location");
    DevGuard g(c->device);
    const int64_t m0 = c->m, m1 = m0 + m_new;
    int rc = grow_storage(c, m1);
    if (rc != FC_OK) return rc;
    const int64_t n_in = (m_new + 63) / 64;
    const uint64_t *src = bitmaps;
    cudaError_t e = cudaSuccess;
    if (where == FC_HOST) {
        const size_t bytes = sizeof(uint64_t) * (size_t)c->R * n_in;
        e = c->io[2].ensure(bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->io[2].p, bitmaps, bytes, cudaMemcpyHostToDevice, c->stream);
        src = (const uint64_t *)c->io[2].p;
    }
    if (e == cudaSuccess) e = launch_append_bits(c->d_bits, c->wstride, c->R, m0, src, n_in, m_new, c->d_marg, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fc_append_bits");
    return finish_append(c, m1);
}

extern "C" int64_t fc_info(const fc_ctx *c, int32_t key)
{
    if (!c) return -1;
    switch (key) {
    case 0: return c->n;
    case 1: return c->m;
    case 2: return c->R;
    case 3: return c->device;
    case 4: return capacity_rows(c);
    case 5: return (int64_t)c->generation;
    case 6: return c->transactions ? 0 : (c->d_D4 && c->opt.codes4) ? 4 : 8;
    case 7: return c->last_batch_on_device;
    default: return -1;
    }
}

extern "C" int fc_marginals(const fc_ctx *c, int64_t *out)
{
    if (!c || !out) return fail(FC_ERR_ARG, "fc_marginals: null argument");
    std::memcpy(out, c->marg.data(), sizeof(int64_t) * c->R);
    return FC_OK;
}

