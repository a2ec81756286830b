// Dedispersion without device allocation.
//
// Some callers cannot allocate device memory at call time: a real-time
// ingest thread must not call cudaMalloc/cudaFree, which can synchronise the
// whole device and take unbounded time, and a process whose device memory is
// already fully reserved by another allocator has none to give.  This entry
// point does the same work as pss_dedisperse but keeps its scratch (the
// kept-channel list, the compacted delay table and the channel-major copy of
// the file) in one file-scope static device array of fixed size, so the only
// device memory it touches is that array and the caller's own input and
// output buffers.
#include <mutex>
#include <string.h>
#include <vector>

#include "pss_internal.h"

namespace pss {

namespace {

// Shared by every call on a device; held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PSS_NOALLOC_SCRATCH_BYTES];
// Error flag the kernels set when they refuse or abandon work.
static __device__ int g_noalloc_err;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};
void* g_err_addr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device (looked up once
// per device; the first call on a device does this set-up).
pss_status scratch_address(int dev, void** out, int** err) {
    if (dev < 0 || dev >= kMaxDevices) return fail(PSS_EINVAL, "pss_dedisperse_noalloc: device index too large");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr, *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        e = cudaGetSymbolAddress(&q, g_noalloc_err);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_err)");
        g_scratch_addr[dev] = p;
        g_err_addr[dev] = q;
    }
    *out = g_scratch_addr[dev];
    *err = (int*)g_err_addr[dev];
    return PSS_OK;
}

}  // namespace

}  // namespace pss

using namespace pss;

extern "C" pss_status pss_dedisperse_noalloc(const pss_plan* plan, const pss_fil_desc* fil, const void* data_dev,
                                             int64_t dm_begin, int64_t dm_end, int32_t* out, void* stream) {
    if (!plan || !fil || !data_dev) return fail(PSS_EINVAL, "pss_dedisperse_noalloc: null plan, descriptor or data");
    if (plan->nsub > 0) return fail(PSS_EINVAL, "pss_dedisperse_noalloc: two-stage (subband) plans are not supported");
    if (fil->nchan != plan->nchan || fil->nsamp != plan->nsamp)
        return fail(PSS_EINVAL, "pss_dedisperse_noalloc: descriptor does not match the plan");
    if (fil->nbits != 8 && fil->nbits != 1) return fail(PSS_EINVAL, "pss_dedisperse_noalloc: nbits must be 8 or 1");
    if (fil->nbits == 1 && fil->nchan % 8) return fail(PSS_EINVAL, "pss_dedisperse_noalloc: 1-bit needs nchan % 8 == 0");
    if (fil->layout != 0 && !(fil->layout == 1 && fil->nbits == 8))
        return fail(PSS_EINVAL, "pss_dedisperse_noalloc: bad layout");
    if (dm_begin < 0 || dm_end > plan->ndm() || dm_begin > dm_end)
        return fail(PSS_EINVAL, "pss_dedisperse_noalloc: DM range outside the plan");
    if (dm_end == dm_begin) return PSS_OK;
    if (!out) return fail(PSS_EINVAL, "pss_dedisperse_noalloc: null out");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    PSS_CUDA(cudaGetDevice(&dev));

    // kept channels and their delays for [dm_begin, dm_end)
    std::vector<int32_t> keep;
    for (int c = 0; c < fil->nchan; ++c)
        if (!fil->chan_mask || fil->chan_mask[c]) keep.push_back(c);
    const int32_t ck = (int32_t)keep.size();
    if (ck == 0) return fail(PSS_EINVAL, "pss_dedisperse_noalloc: channel mask removes every channel");
    const int64_t ndm = dm_end - dm_begin;
    const int TN = dedisp_tile_samples();
    const int64_t pitch = ((fil->nsamp + TN + 256) + 63) / 64 * 64;
    const size_t table_bytes = ((size_t)(ck + ndm * ck) * sizeof(int32_t) + 255) / 256 * 256;
    const size_t need = table_bytes + (size_t)ck * pitch + 64;
    if (need > (size_t)PSS_NOALLOC_SCRATCH_BYTES)
        return fail(PSS_EINVAL, "pss_dedisperse_noalloc: needs " + std::to_string(need) +
                                    " bytes of scratch; the static array holds " +
                                    std::to_string((size_t)PSS_NOALLOC_SCRATCH_BYTES) +
                                    " (use pss_dedisperse, or fewer channels, samples or DM trials)");
    void* base = nullptr;
    int* d_err = nullptr;
    PSS_TRY(scratch_address(dev, &base, &d_err));
    int32_t* d_keep = (int32_t*)base;
    uint8_t* d_xcm = (uint8_t*)base + table_bytes;

    std::vector<int32_t> host((size_t)ck * (1 + ndm));
    memcpy(host.data(), keep.data(), sizeof(int32_t) * ck);
    for (int64_t i = 0; i < ndm; ++i)
        for (int32_t r = 0; r < ck; ++r)
            host[(size_t)ck * (1 + i) + r] = plan->delays[(size_t)(dm_begin + i) * plan->nchan + keep[r]];

    // every launch's delay spread, checked against the kernel's limits before any work is enqueued,
    // so that a refused request leaves nothing running on the stream
    struct Launch {
        int64_t b0;
        int32_t nb, spread;
        const StageInfo* st;
    };
    std::vector<Launch> launches;
    for (size_t si = 0; si < plan->stages.size(); ++si) {
        const StageInfo& st = plan->stages[si];
        const int64_t lo = std::max<int64_t>(dm_begin, st.first);
        const int64_t hi = std::min<int64_t>(dm_end, st.first + st.n_dm);
        for (int64_t b0 = lo; b0 < hi; b0 += 1024) {
            const int32_t nb = (int32_t)std::min<int64_t>(1024, hi - b0);
            const int32_t* hrow = host.data() + (size_t)ck * (1 + (b0 - dm_begin));
            // largest delay spread over the kernel's groups of consecutive trials
            const int32_t G = dedisp_group_trials();
            int32_t spread = 0;
            for (int32_t g = 0; g < nb; g += G)
                for (int32_t c = 0; c < ck; ++c) {
                    int32_t mn = hrow[(size_t)g * ck + c], mx = mn;
                    for (int32_t i = g + 1; i < std::min(nb, g + G); ++i) {
                        mn = std::min(mn, hrow[(size_t)i * ck + c]);
                        mx = std::max(mx, hrow[(size_t)i * ck + c]);
                    }
                    spread = std::max(spread, mx - mn);
                }
            if (!dedisp_launch_fits(spread, ck, 0))
                return fail(PSS_EINVAL, "pss_dedisperse_noalloc: the delay spread of 16 consecutive trials (" +
                                            std::to_string(spread) + " samples) is too large for the kernel");
            launches.push_back({b0, nb, spread, &st});
        }
    }

    // from the first enqueued operation on, every exit waits for the stream: nothing of this call
    // may still be writing into `out` or the shared scratch when it returns
    auto enqueue = [&]() -> pss_status {
        PSS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
        PSS_CUDA(cudaMemcpyAsync(d_keep, host.data(), host.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));

        PrepArgs pa;
        pa.src = (const uint8_t*)data_dev;
        pa.nchan = fil->nchan;
        pa.nbits = fil->nbits;
        pa.layout = fil->layout;
        pa.nsamp = fil->nsamp;
        pa.keep = d_keep;
        pa.ck = ck;
        pa.xcm = d_xcm;
        pa.pitch = pitch;
        PSS_CUDA(launch_prep(pa, s));
        int64_t off = 0;
        for (const Launch& l : launches) {
            DedispArgs da{};
            da.xcm = d_xcm;
            da.pitch = pitch;
            da.ck = ck;
            da.delays = d_keep + (size_t)ck * (1 + (l.b0 - dm_begin));
            da.nb = l.nb;
            da.nv = l.st->nv;
            da.ds = l.st->ds;
            da.out_f = nullptr;
            da.out_i = out + off;
            da.out_stride = l.st->nv;
            da.sums = nullptr;
            da.spread = l.spread;
            da.err = d_err;
            PSS_CUDA(launch_dedisp(da, 0, s));
            off += (int64_t)l.nb * l.st->nv;
        }
        return PSS_OK;
    };
    const pss_status st = enqueue();
    if (st != PSS_OK) {
        cudaStreamSynchronize(s);  // the error is already recorded; this only drains the stream
        return st;
    }
    int flag = 0;
    PSS_CUDA(cudaMemcpyAsync(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    // the delay upload reads `host`, which goes out of scope on return
    PSS_CUDA(cudaStreamSynchronize(s));
    if (flag) return fail(flag == 1 ? PSS_ETIMEOUT : PSS_EINVAL, "pss_dedisperse_noalloc: the kernel refused or abandoned its work");
    return PSS_OK;
}
