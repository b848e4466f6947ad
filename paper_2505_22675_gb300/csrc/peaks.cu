// bg_alu_peak: the ALU peaks of this GPU, measured, for the roofline of the
// kernels that no memory or tensor-core bound describes (the k-NN's integer
// work, the kriging solve's FP32 arithmetic, the FP64 pipe).
//
// Each thread runs eight independent dependency chains of one instruction
// kind, so every SM sub-partition always has an issuable instruction of that
// kind; the grid holds two 1024-thread blocks per SM. Thread 0 of every block
// reads the SM clock counter (clock64) and the global nanosecond timer at its
// start and end, so the call also returns the SM clock the kernel ran at:
// a peak per SM cycle that does not assume the maximum clock.
#include <algorithm>
#include <vector>

#include "bg_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 1024;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// kind 0: a = a * b + c (FP32 FMA); 1: a = a * m + c (INT32 IMAD);
// 2: a = (a + b) ^ c (INT32 add, then xor); 3: a = a * b + c (FP64 FMA)
template <int kKind>
__global__ void __launch_bounds__(kPeakThreads, 2)
    k_alu_peak(long long iters, unsigned seed, int store, unsigned long long* sink,
               unsigned long long* clk) {
    unsigned long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        t0 = global_ns();
        c0 = clock64();
    }
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long out = 0;
    if constexpr (kKind == 0) {
        float a[kChains];
        const float b = 0.9999f + 1e-9f * (float)(seed & 7), c = 1e-6f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = (float)(tid + i) * 1e-7f;
#pragma unroll 4
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out = __float_as_uint(s);
    } else if constexpr (kKind == 1) {
        unsigned a[kChains];
        const unsigned m = 2 * seed + 1, c = seed ^ 0x9e3779b9u;
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = tid * 8 + i;
#pragma unroll 4
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = a[i] * m + c;
        unsigned s = 0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s ^= a[i];
        out = s;
    } else if constexpr (kKind == 2) {
        unsigned a[kChains];
        const unsigned b = seed | 1, c = seed * 0x85ebca6bu;
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = tid * 8 + i;
#pragma unroll 4
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = (a[i] + b) ^ c;
        unsigned s = 0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out = s;
    } else {
        double a[kChains];
        const double b = 0.9999 + 1e-12 * (double)(seed & 7), c = 1e-9;
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = (double)(tid + i) * 1e-9;
#pragma unroll 2
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out = (unsigned long long)__double_as_longlong(s);
    }
    // the caller passes store = 0, but the compiler cannot know it: the
    // chains' results stay live
    if (store) sink[0] = out;
    if (threadIdx.x == 0) {
        const unsigned long long c1 = clock64(), t1 = global_ns();
        clk[2 * blockIdx.x] = c1 - c0;
        clk[2 * blockIdx.x + 1] = t1 - t0;
    }
}

template <int kKind>
bg_status run_peak(int blocks, long long iters, cudaStream_t st, unsigned long long* sink,
                   unsigned long long* clk, float* ms) {
    cudaEvent_t e0, e1;
    BG_CUDA(cudaEventCreate(&e0));
    BG_CUDA(cudaEventCreate(&e1));
    BG_CUDA(cudaEventRecord(e0, st));
    k_alu_peak<kKind><<<blocks, kPeakThreads, 0, st>>>(iters, 12345u, 0, sink, clk);
    bg::note_launches(1);
    BG_CUDA(cudaGetLastError());
    BG_CUDA(cudaEventRecord(e1, st));
    BG_CUDA(cudaEventSynchronize(e1));
    BG_CUDA(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return BG_OK;
}

bg_status run_kind(int kind, int blocks, long long iters, cudaStream_t st,
                   unsigned long long* sink, unsigned long long* clk, float* ms) {
    switch (kind) {
        case 0: return run_peak<0>(blocks, iters, st, sink, clk, ms);
        case 1: return run_peak<1>(blocks, iters, st, sink, clk, ms);
        case 2: return run_peak<2>(blocks, iters, st, sink, clk, ms);
        default: return run_peak<3>(blocks, iters, st, sink, clk, ms);
    }
}

// operations one loop iteration of one chain counts (an FMA is 2 flops; the
// add-then-xor step is 2 integer operations)
double ops_per_step(int kind) { return kind == 1 ? 1.0 : 2.0; }

}  // namespace

extern "C" bg_status bg_alu_peak(int device, int kind, double* ops_per_s, double* sm_mhz_out) {
    using namespace bg;
    if (kind < 0 || kind > 3 || !ops_per_s) {
        set_error("kind must be 0..3 and ops_per_s not NULL");
        return BG_ERR_INVALID_ARG;
    }
    int prev = 0;
    BG_CUDA(cudaGetDevice(&prev));
    BG_CUDA(cudaSetDevice(device));
    int sms = 0;
    BG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = 2 * sms;
    cudaStream_t st = nullptr;
    unsigned long long* buf = nullptr;
    bg_status rc = BG_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        rc = cuda_fail(e, what);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) fail(e, "cudaStreamCreate");
    if (rc == BG_OK) {
        e = cudaMalloc(&buf, sizeof(unsigned long long) * (1 + 2 * (size_t)blocks));
        if (e != cudaSuccess) fail(e, "cudaMalloc");
    }
    double best = 0.0, mhz = 0.0;
    if (rc == BG_OK) {
        // calibrate the loop length to about 100 ms, then keep the best of three
        float ms = 0.0f;
        long long iters = kind == 3 ? 256 : 4096;
        rc = run_kind(kind, blocks, iters, st, buf, buf + 1, &ms);
        if (rc == BG_OK && ms > 0.0f)
            iters = std::max<long long>(iters, (long long)(iters * (100.0 / ms)));
        for (int rep = 0; rep < 3 && rc == BG_OK; ++rep) {
            rc = run_kind(kind, blocks, iters, st, buf, buf + 1, &ms);
            if (rc != BG_OK) break;
            const double ops = ops_per_step(kind) * kChains * (double)iters * blocks * kPeakThreads;
            const double rate = ops / (ms * 1e-3);
            if (rate > best) {
                best = rate;
                std::vector<unsigned long long> h(2 * (size_t)blocks);
                e = cudaMemcpy(h.data(), buf + 1, h.size() * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) {
                    fail(e, "cudaMemcpy");
                    break;
                }
                std::vector<double> f;
                for (int b = 0; b < blocks; ++b)
                    if (h[2 * b + 1] > 0) f.push_back(1e3 * (double)h[2 * b] / (double)h[2 * b + 1]);
                if (!f.empty()) {
                    std::nth_element(f.begin(), f.begin() + f.size() / 2, f.end());
                    mhz = f[f.size() / 2];
                }
            }
        }
    }
    if (buf) cudaFree(buf);
    if (st) cudaStreamDestroy(st);
    cudaSetDevice(prev);
    if (rc != BG_OK) return rc;
    *ops_per_s = best;
    if (sm_mhz_out) *sm_mhz_out = mhz;
    return BG_OK;
}
