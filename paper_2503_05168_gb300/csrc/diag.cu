// diag.cu -- measured issue peaks of the pipes the rasterizer runs on, and the
// look-back scan on caller memory (with a test hook for its bounded wait).
//
// Peaks: each kernel keeps every scheduler of every SM busy with independent
// dependency chains of one instruction kind -- FP32 fused multiply-add (FMA
// pipe), ex2.approx (the MUFU / XU pipe), float min/max and integer logic (the
// ALU pipe) -- and the lane-operations per second follow from CUDA-event
// times.  The blending of Sec. 3.1 Eqns. 1-2 and Alg. 1 is bound by these
// pipes, not by memory, so its roofline divides by these rates.
#include <algorithm>
#include <atomic>

#include "kernels.h"
#include "seele.h"

namespace seele {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ float peak_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- x a + b on kChains independent chains; 16 steps per loop trip.
__global__ void __launch_bounds__(kPeakThreads) peak_ffma_kernel(float a, float b, int trips, float* sink) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[0] = s;  // never true; keeps the chains live
}

// x <- 2^(-x) on kChains chains (x stays in [0.5, 1]); 8 steps per trip.
__global__ void __launch_bounds__(kPeakThreads) peak_ex2_kernel(float a, int trips, float* sink) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 0.5f + 1e-4f * (float)(threadIdx.x + k);
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = peak_ex2(x[k] * a);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[0] = s;
}

// x <- min(max(x, lo_u), hi_u) with sixteen different runtime bounds per trip.
__global__ void __launch_bounds__(kPeakThreads) peak_fmnmx_kernel(const float* __restrict__ bounds, int trips,
                                                                 float* sink) {
    float lo[16], hi[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        lo[u] = __ldg(bounds + u);
        hi[u] = __ldg(bounds + 16 + u);
    }
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)threadIdx.x + 0.1f * (float)k;
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fminf(fmaxf(x[k], lo[u]), hi[u]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[0] = s;
}

__device__ __forceinline__ uint32_t lop3_xor_and_or(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;  // (a ^ b) & (a | c): truth table 0x38 on (0xf0, 0xcc, 0xaa)
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x38;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// x <- (x ^ p_u) & (x | q_u): one three-input logic instruction per step.
__global__ void __launch_bounds__(kPeakThreads) peak_lop3_kernel(uint32_t p, uint32_t q, int trips,
                                                                uint32_t* sink) {
    uint32_t x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 2654435761u + (uint32_t)k;
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = lop3_xor_and_or(x[k], p + 977u * u, q ^ (6151u * u));
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= x[k];
    if (s == 0x9e3779b9u) sink[0] = s;
}

template <typename F>
float best_ms(cudaStream_t s, F launch) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    launch();  // warm-up (clocks, instruction cache)
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a, s);
        launch();
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            best = -1.f;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

std::atomic<uint32_t> g_scan_epoch{1};

}  // namespace
}  // namespace seele

using namespace seele;

extern "C" seele_status seele_measure_peaks(int device, void* cuda_stream, seele_peaks* out) {
    if (!out) return SEELE_ERR_ARG;
    *out = seele_peaks{};
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        (void)cudaGetLastError();
        return SEELE_ERR_ARG;
    }
    int sms = 0, clock_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, device);
    out->sm_count = sms;
    out->sm_clock_max_mhz = clock_khz / 1000;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // 32 floats of bounds and one sink word: the only device memory used
    void* mem = nullptr;
    if (cudaMalloc(&mem, 256) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaSetDevice(prev);
        return SEELE_ERR_OOM;
    }
    float hb[32];
    for (int u = 0; u < 16; ++u) {
        hb[u] = -4.f + 0.01f * u;       // lower bounds, below every chain value
        hb[16 + u] = 4.f - 0.01f * u;   // upper bounds, above it
    }
    cudaMemcpy(mem, hb, sizeof hb, cudaMemcpyHostToDevice);
    float* fb = static_cast<float*>(mem);
    float* sink = fb + 32;
    uint32_t* isink = reinterpret_cast<uint32_t*>(fb + 40);
    const dim3 grid(sms * 8), block(kPeakThreads);  // 2048 threads on every SM
    const double threads = (double)grid.x * kPeakThreads;
    const int t_fma = 2048, t_ex2 = 512, t_mm = 512, t_lop = 1024;
    out->fp32_ms = best_ms(s, [&] { peak_ffma_kernel<<<grid, block, 0, s>>>(0.999f, 1e-3f, t_fma, sink); });
    out->sfu_ms = best_ms(s, [&] { peak_ex2_kernel<<<grid, block, 0, s>>>(-1.f, t_ex2, sink); });
    out->alu_fmnmx_ms = best_ms(s, [&] { peak_fmnmx_kernel<<<grid, block, 0, s>>>(fb, t_mm, sink); });
    out->alu_lop3_ms = best_ms(s, [&] {
        peak_lop3_kernel<<<grid, block, 0, s>>>(0x5bd1e995u, 0x00010200u, t_lop, isink);
    });
    const cudaError_t e = cudaGetLastError();
    cudaFree(mem);
    cudaSetDevice(prev);
    if (e != cudaSuccess || out->fp32_ms <= 0.f || out->sfu_ms <= 0.f || out->alu_fmnmx_ms <= 0.f ||
        out->alu_lop3_ms <= 0.f)
        return SEELE_ERR_CUDA;
    out->fp32_tops = threads * kChains * 16.0 * t_fma / (out->fp32_ms * 1e-3) / 1e12;
    out->sfu_tops = threads * kChains * 8.0 * t_ex2 / (out->sfu_ms * 1e-3) / 1e12;
    out->alu_fmnmx_tops = threads * kChains * 32.0 * t_mm / (out->alu_fmnmx_ms * 1e-3) / 1e12;
    out->alu_lop3_tops = threads * kChains * 16.0 * t_lop / (out->alu_lop3_ms * 1e-3) / 1e12;
    return SEELE_OK;
}

extern "C" size_t seele_scan_scratch_bytes(uint32_t n) {
    return 256 + 8ull * exclusive_scan_blocks(n);
}

extern "C" seele_status seele_exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, void* scratch,
                                             uint32_t withhold_block, uint32_t spin_limit, void* cuda_stream) {
    if (n > 0 && (!in || !out)) return SEELE_ERR_ARG;
    if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 255u) || (reinterpret_cast<uintptr_t>(in) & 15u))
        return SEELE_ERR_ARG;
    if (n == 0) return SEELE_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    DeviceStatus* st = reinterpret_cast<DeviceStatus*>(base);
    uint64_t* lookback = reinterpret_cast<uint64_t*>(base + 256);
    // the status word, its tickets and every look-back entry start cleared
    if (cudaMemsetAsync(scratch, 0, seele_scan_scratch_bytes(n), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return SEELE_ERR_CUDA;
    }
    launch_exclusive_scan(in, n, out, lookback, g_scan_epoch.fetch_add(1), st, 0, s, spin_limit, withhold_block);
    int32_t err = 0;
    if (cudaPeekAtLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(&err, base, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        return SEELE_ERR_CUDA;
    }
    if (err == kOk) return SEELE_OK;
    return err == kErrTimeout ? SEELE_ERR_TIMEOUT : SEELE_ERR_INTERNAL;
}
