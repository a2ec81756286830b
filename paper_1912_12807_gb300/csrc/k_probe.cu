// Measured instruction throughputs of the device: the denominators of the
// integer and FP32 rooflines (the dedispersion sums and the template
// correlation), taken by timing long runs of one instruction kind instead
// of deriving them from lane counts.
//
// Each probe kernel runs one wave of CTAs (4 per SM, 256 threads) whose
// threads advance 8 independent chains for `iters` x 16 steps, each step one
// instruction of the kind probed, written as inline PTX so the compiler does
// not fold the chains:
//   0  add3   a = a + b + c        (two 32-bit additions: IADD3)
//   1  lop3   a = (a & b) ^ c      (one three-input logic op)
//   2  prmt   a = byte_perm(a, b)  (one byte permute)
//   3  imad   a = a * b + c        (one integer multiply-add)
//   4  ffma   a = a * b + c        (FP32 fused multiply-add: 2 flops)
//   5  mix    lop3 and imad alternating (the issue rate when both the integer
//             and the FMA pipes are busy)
//   6  lds    32-bit shared-memory loads, conflict-free, each folded into
//             its chain by an add (shared-memory words per clock)
// Each CTA's thread 0 records the SM cycles its loop took (clock64); the
// rate per SM clock is the work of an SM's CTAs over the longest of them,
// and the rate per second uses the CUDA-event time of the launch.
#include "pss_internal.h"

namespace pss {

namespace {

constexpr int PNT = 256;
constexpr int PCTA_PER_SM = 4;
constexpr int PUNROLL = 16;

template <int OP>
__global__ void __launch_bounds__(PNT) k_probe(uint32_t* sink, int iters, uint32_t s0,
                                               unsigned long long* cycles) {
    __shared__ uint32_t lds[PNT * 2];
    uint32_t a[8];
    float f[8];
    const uint32_t b = s0 ^ (uint32_t)threadIdx.x, c = s0 * 3u + (uint32_t)blockIdx.x;
    const float fb = 1.0f - 1e-7f * (float)(threadIdx.x & 7), fc = 1e-9f * (float)(blockIdx.x & 15);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = (uint32_t)threadIdx.x * (uint32_t)(i + 1) + s0;
        f[i] = (float)a[i] * 1e-6f;
    }
    if (OP == 6) {
        for (int i = threadIdx.x; i < PNT * 2; i += PNT) lds[i] = (uint32_t)i * 2654435761u ^ s0;
        __syncthreads();
    }
    const uint32_t lds_base = (uint32_t)__cvta_generic_to_shared(lds) + 4u * (uint32_t)threadIdx.x;
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < PUNROLL; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (OP == 0) {
                    asm volatile("add.u32 %0, %0, %1;\n\tadd.u32 %0, %0, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
                } else if (OP == 1) {
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x6a;" : "+r"(a[i]) : "r"(b), "r"(c));
                } else if (OP == 2) {
                    asm volatile("prmt.b32 %0, %0, %1, 0x5140;" : "+r"(a[i]) : "r"(b));
                } else if (OP == 3) {
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
                } else if (OP == 4) {
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[i]) : "f"(fb), "f"(fc));
                } else if (OP == 5) {
                    if (i & 1) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
                    else asm volatile("lop3.b32 %0, %0, %1, %2, 0x6a;" : "+r"(a[i]) : "r"(b), "r"(c));
                } else {
                    // word (tid + 256*(i & 1)) of the table: consecutive lanes, consecutive words
                    uint32_t w;
                    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(w) : "r"(lds_base + 1024u * (uint32_t)(i & 1)));
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(w));
                }
            }
        }
    }
    const long long t1 = clock64();
    uint32_t acc = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= a[i] ^ __float_as_uint(f[i]);
    if (acc == 0x9e3779b9u) sink[blockIdx.x * PNT + threadIdx.x] = acc;  // keeps the chains live
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

template <int OP>
cudaError_t run_probe(int sms, int iters, uint32_t* sink, unsigned long long* cyc, cudaStream_t s, float* ms,
                      unsigned long long* cycles) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    const int grid = sms * PCTA_PER_SM;
    k_probe<OP><<<grid, PNT, 0, s>>>(sink, iters / 8 + 1, 1u, cyc);  // warm
    e = cudaMemsetAsync(cyc, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_probe<OP><<<grid, PNT, 0, s>>>(sink, iters, 7u, cyc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(cycles, cyc, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

cudaError_t probe_peaks(int sms, cudaStream_t s, uint32_t* sink, unsigned long long* cyc, double per_clk[7],
                        double per_s[7], double* sm_mhz) {
    // operations per probe step and thread (instructions, except add3: 2 additions, ffma: 2 flops,
    // lds: 4 bytes)
    const double per_step[7] = {2.0, 1.0, 1.0, 1.0, 2.0, 1.0, 4.0};
    const int iters = 4096;
    double mhz_sum = 0.0;
    for (int op = 0; op < 7; ++op) {
        float ms = 0.f;
        unsigned long long cycles = 0;
        cudaError_t e;
        switch (op) {
            case 0: e = run_probe<0>(sms, iters, sink, cyc, s, &ms, &cycles); break;
            case 1: e = run_probe<1>(sms, iters, sink, cyc, s, &ms, &cycles); break;
            case 2: e = run_probe<2>(sms, iters, sink, cyc, s, &ms, &cycles); break;
            case 3: e = run_probe<3>(sms, iters, sink, cyc, s, &ms, &cycles); break;
            case 4: e = run_probe<4>(sms, iters, sink, cyc, s, &ms, &cycles); break;
            case 5: e = run_probe<5>(sms, iters, sink, cyc, s, &ms, &cycles); break;
            default: e = run_probe<6>(sms, iters, sink, cyc, s, &ms, &cycles); break;
        }
        if (e != cudaSuccess) return e;
        const double ops_per_sm = (double)PCTA_PER_SM * PNT * iters * PUNROLL * 8 * per_step[op];
        per_clk[op] = cycles ? ops_per_sm / (double)cycles : 0.0;
        per_s[op] = ms > 0.f ? ops_per_sm * sms / (ms * 1e-3) : 0.0;
        mhz_sum += ms > 0.f ? (double)cycles / (ms * 1e3) : 0.0;
    }
    *sm_mhz = mhz_sum / 7.0;
    return cudaSuccess;
}

}  // namespace pss

extern "C" pss_status pss_measure_peaks(int device, pss_peaks* out) {
    using namespace pss;
    if (!out) return fail(PSS_EINVAL, "pss_measure_peaks: null out");
    int n = 0;
    PSS_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(PSS_EINVAL, "pss_measure_peaks: no such device");
    PSS_CUDA(cudaSetDevice(device));
    int sms = 0;
    PSS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    cudaStream_t s = nullptr;
    PSS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    void* buf = nullptr;
    const size_t sink_bytes = (size_t)sms * 4 * 256 * sizeof(uint32_t);
    cudaError_t e = cudaMalloc(&buf, sink_bytes + 256);
    double per_clk[7] = {0}, per_s[7] = {0}, mhz = 0.0;
    if (e == cudaSuccess)
        e = probe_peaks(sms, s, (uint32_t*)buf, (unsigned long long*)((char*)buf + sink_bytes), per_clk, per_s, &mhz);
    if (buf) cudaFree(buf);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_fail(e, "pss_measure_peaks");
    out->sms = sms;
    out->sm_mhz = mhz;
    out->add3_per_clk_sm = per_clk[0];
    out->lop3_per_clk_sm = per_clk[1];
    out->prmt_per_clk_sm = per_clk[2];
    out->imad_per_clk_sm = per_clk[3];
    out->ffma_flops_per_clk_sm = per_clk[4];
    out->mix_per_clk_sm = per_clk[5];
    out->lds_bytes_per_clk_sm = per_clk[6];
    out->int32_adds_per_s = per_s[0];
    out->lop3_per_s = per_s[1];
    out->prmt_per_s = per_s[2];
    out->imad_per_s = per_s[3];
    out->fp32_flops_per_s = per_s[4];
    out->mix_per_s = per_s[5];
    out->lds_bytes_per_s = per_s[6];
    return PSS_OK;
}
