// sf_noalloc.cu -- rotation (automorphism + key switching) that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: code running inside a stream-ordered
// allocator's or a host framework's memory budget that must not grow, plug-ins
// loaded into a process whose allocator owns the whole device, and real-time
// paths where an allocation (or the synchronising cudaFree that a growing
// workspace implies) would stall.  sf_rotate_noalloc serves them: its scratch
// is the fixed array below, reserved once per GPU when the library's module
// is loaded on that GPU, and every call reuses it.
#include <algorithm>
#include <mutex>

#include "sf_internal.h"
#include "sf_ks.h"

// 32 MiB of scratch per GPU that loads this library, held until the process exits.
#define SF_NOALLOC_SCRATCH_WORDS ((size_t)4 << 20)
static __device__ __align__(256) u64 g_sf_noalloc_scratch[SF_NOALLOC_SCRATCH_WORDS];

#define SF_NOALLOC_MAX_DEVICES 64
static u64 *g_noalloc_ptr[SF_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// Device address of the array on `device` (which must be current).  In host
// code the array's name is only a host-side stand-in, so the address has to
// come from cudaGetSymbolAddress, once per device.
static sf_status noalloc_scratch(int device, u64 **out)
{
    if (device < 0 || device >= SF_NOALLOC_MAX_DEVICES) return sf_set_error(SF_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sf_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return sf_set_error(SF_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorString(e));
        g_noalloc_ptr[device] = (u64 *)p;
    }
    *out = g_noalloc_ptr[device];
    return SF_OK;
}

static inline size_t round_words(size_t w) { return (w + 31) & ~(size_t)31; }

extern "C" sf_status sf_rotate_noalloc(sf_ctx *ctx, const sf_rotkeys *rk, int32_t d, const uint64_t *d_ct,
                                       uint64_t *d_out, int32_t count, void *stream)
{
    if (!ctx) return sf_set_error(SF_EINVAL, "sf_rotate_noalloc: null context");
    SF_CUDA_TRY(cudaSetDevice(ctx->device));
    const SfRing &R = ctx->ring;
    if (!rk || rk->ctx != ctx || !d_ct || !d_out || count < 1) return sf_set_error(SF_EINVAL, "sf_rotate_noalloc: bad arguments");
    int slot = -1;
    for (size_t t = 0; t < rk->d.size(); ++t)
        if (rk->d[t] == d) slot = (int)t;
    if (slot < 0) return sf_set_error(SF_EINVAL, "no rotation key for d = %d", d);
    const size_t ct = (size_t)2 * R.L * R.n;
    // key switches run in launch batches of the context's size, as in sf_rotate
    const int batch = std::min(ctx->ks_batch, (int)count);
    const size_t need = 2 * round_words((size_t)count * ct) + round_words(sf_ks_scratch_words(R) * batch);
    if (need > SF_NOALLOC_SCRATCH_WORDS)
        return sf_set_error(SF_EINVAL,
                            "sf_rotate_noalloc: %d ciphertexts need %zu bytes of scratch, the fixed maximum is %zu bytes",
                            count, need * sizeof(u64), SF_NOALLOC_SCRATCH_WORDS * sizeof(u64));
    u64 *ws = nullptr;
    SF_TRY(noalloc_scratch(ctx->device, &ws));
    cudaStream_t st = (cudaStream_t)stream;
    u64 *in_ntt = ws, *out_ntt = ws + round_words((size_t)count * ct);
    u64 *ks = out_ntt + round_words((size_t)count * ct);
    // per-launch event bracketing would create CUDA events; keep this call free of that
    const int timing = ctx->kernel_timing;
    ctx->kernel_timing = 0;
    sf_status s = SF_OK;
    {
        SfPolyJob jobs[64];
        for (int x0 = 0; x0 < count * 2 * R.L && s == SF_OK; x0 += 64) {
            int cnt = 0;
            for (int x = x0; x < count * 2 * R.L && cnt < 64; ++x, ++cnt)
                jobs[cnt] = {d_ct + (size_t)x * R.n, in_ntt + (size_t)x * R.n, x % R.L};
            s = sf_ntt_jobs(ctx, jobs, cnt, false, st);
        }
        if (s == SF_OK) {
            SfKsBatch b;
            memset(&b, 0, sizeof(b));
            b.E = in_ntt;
            b.E_stride = ct;
            b.out = out_ntt;
            b.out_stride = ct;
            b.inner = 1 << 30;
            b.count = count;
            b.d = d;
            b.add_v = 0;
            b.key = rk->d_keys + rk->key_words * slot;
            s = sf_ks_run(ctx, b, ks, batch, st);
        }
        for (int x0 = 0; x0 < count * 2 * R.L && s == SF_OK; x0 += 64) {
            int cnt = 0;
            for (int x = x0; x < count * 2 * R.L && cnt < 64; ++x, ++cnt)
                jobs[cnt] = {out_ntt + (size_t)x * R.n, d_out + (size_t)x * R.n, x % R.L};
            s = sf_ntt_jobs(ctx, jobs, cnt, true, st);
        }
    }
    ctx->kernel_timing = timing;
    return s;
}
