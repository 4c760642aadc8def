// Instruction-rate microbenchmark of the arithmetic the filter kernels issue:
// FP32 FMA (fma.rn.f32), two-lane FP32 FMA (fma.rn.f32x2), the exponent
// (ex2.approx.ftz.f32, ex2.approx.f16x2), the four-byte integer dot product
// (dp4a.s32.s32) and the mixed loop of one filter tap pair in the paired
// expanded form (per output pixel one dp4a of the packed colours, then one
// two-lane FMA for the two pixels' exponents, one ex2 per pixel and two
// two-lane FMA into numerator and weight sum: 3.5 instructions a tap), FP32
// adds into shared memory (the scatter form's accumulation), half2 FMA
// (fma.rn.f16x2) and the FP16 form's tap pair (half2 colour differences,
// squared distance and exponent for two output rows, one ex2.approx.f16x2, the
// weights widened to FP32 and accumulated). Its measured rates are the peaks
// the filter rooflines divide by.
//
// Every thread runs kChains independent dependency chains, unrolled, so that
// issue (not latency) limits the rate once enough warps are resident; each
// thread stores one word at the end so that nothing is eliminated. The ex2
// chains feed every result back into the next exponent: values run to +inf
// after a few steps and stay there (the instruction's rate does not depend on
// its operand).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

enum Op {
    OP_FFMA = 0, OP_FFMA2 = 1, OP_EX2 = 2, OP_EX2_H2 = 3, OP_TAP_PAIRED = 4, OP_RED_SHARED = 5, OP_HFMA2 = 6,
    OP_TAP_FP16 = 7, OP_DP4A = 8, OP_COUNT = 9
};

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t ex2h2(uint32_t x) {
    uint32_t y;
    asm("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(kThreads, 6) rate_kernel(float *__restrict__ out, int iters, float s) {
    const int tid = blockIdx.x * kThreads + threadIdx.x;
    float sink = 0.0f;
    if (OP == OP_FFMA) {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = s + 0.001f * c + 1e-7f * tid;
        const float m = 0.9999f - 1e-9f * s, k = 1e-4f + 1e-9f * s;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) sink += a[c];
    } else if (OP == OP_FFMA2) {
        float2 a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = make_float2(s + 0.001f * c, s - 0.001f * c + 1e-7f * tid);
        const float2 m = make_float2(0.9999f - 1e-9f * s, 0.9998f), k = make_float2(1e-4f, 2e-4f + 1e-9f * s);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, k);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) sink += a[c].x + a[c].y;
    } else if (OP == OP_EX2) {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = -s - 0.01f * c - 1e-7f * tid;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) a[c] = ex2f(a[c]);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) sink += a[c];
    } else if (OP == OP_EX2_H2) {
        uint32_t a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 0xBC00BC00u ^ (uint32_t)(c + (tid & 7));   // about (-1, -1)
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) a[c] = ex2h2(a[c]);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) sink += __uint_as_float(a[c] & 0x3FFFFFFFu);
    } else if (OP == OP_DP4A) {
        int a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = (int)(0x01020304u * (uint32_t)(c + 1)) ^ tid;
        const int m = (int)(0x7F01FF80u ^ (uint32_t)(s * 3.0f));
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) a[c] = __dp4a(a[c], m, a[c]);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) sink += (float)(a[c] & 0xFF);
    } else if (OP == OP_HFMA2) {
        __half2 a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __floats2half2_rn(0.5f + 0.01f * c, 0.25f + 1e-3f * (tid & 15));
        const __half2 m = __floats2half2_rn(0.99f * s, 0.98f), k = __floats2half2_rn(1e-3f, 2e-3f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) a[c] = __hfma2(a[c], m, k);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) sink += __low2float(a[c]) + __high2float(a[c]);
    } else if (OP == OP_TAP_FP16) {   // the FP16 form's tap pair: two output rows of one column, one neighbour
        constexpr int P = kChains / 2;
        __half2 q[P];
        float num[2 * P], den[2 * P];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            q[c] = __floats2half2_rn(3.0f + c, 5.0f + 1e-3f * (tid & 7));
            num[2 * c] = num[2 * c + 1] = den[2 * c] = den[2 * c + 1] = 0.0f;
        }
        const __half2 cr = __floats2half2_rn(1.0f * s, 2.0f), cg = __floats2half2_rn(3.0f, 1.0f),
                      cb = __floats2half2_rn(2.0f, 4.0f), kc2 = __floats2half2_rn(-0.01f, -0.01f),
                      sp = __floats2half2_rn(-0.1f, -0.2f);
        const float qd = 2.5f * s;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const __half2 dr = __hsub2(q[c], cr), dg = __hsub2(q[c], cg), db = __hsub2(q[c], cb);
                    const __half2 n2 = __hfma2(dr, dr, __hfma2(dg, dg, __hmul2(db, db)));
                    uint32_t wb;
                    const __half2 e = __hfma2(n2, kc2, sp);
                    asm("ex2.approx.f16x2 %0, %1;" : "=r"(wb) : "r"(*reinterpret_cast<const uint32_t *>(&e)));
                    const float2 w = __half22float2(*reinterpret_cast<const __half2 *>(&wb));
                    num[2 * c] = fmaf(w.x, qd, num[2 * c]);
                    den[2 * c] += w.x;
                    num[2 * c + 1] = fmaf(w.y, qd, num[2 * c + 1]);
                    den[2 * c + 1] += w.y;
                    q[c] = dr;   // the next neighbour depends on this one (nothing to hoist, no extra instruction)
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 2 * P; ++c) sink += num[c] + den[c];
    } else if (OP == OP_RED_SHARED) {   // FP32 add to shared memory, no return value, distinct words per lane
        __shared__ float acc[kChains][kThreads];
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c][threadIdx.x] = 0.0f;
        __syncthreads();
        const float v = 1e-3f * s;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) atomicAdd(&acc[c][threadIdx.x], v);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kChains; ++c) sink += acc[c][threadIdx.x];
    } else {   // OP_TAP_PAIRED: kChains / 2 independent tap pairs per thread
        constexpr int P = kChains / 2;
        int q0[P], q1[P];
        float2 num[P], den[P];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            q0[c] = 0x4B400000 + c + (tid & 15);
            q1[c] = 0x4B400000 - c;
            num[c] = den[c] = make_float2(0.0f, 0.0f);
        }
        const int cp0 = (int)(0x00102030u ^ (uint32_t)s), cp1 = 0x00F0E0D0;
        const float2 kc2 = make_float2(1e-3f, 1e-3f), bias = make_float2(-12582.9f * s, -12582.8f);
        const float2 g = make_float2(1.5f, 2.5f), f = make_float2(0.75f, 0.5f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    // colour dot products of two output pixels at one tap, read as biased floats
                    q0[c] = __dp4a(cp0, q0[c], 0x4B400000);
                    q1[c] = __dp4a(cp1, q1[c], 0x4B400000);
                    // both exponents: one two-lane FMA
                    const float2 x = __ffma2_rn(make_float2(__int_as_float(q0[c]), __int_as_float(q1[c])), kc2, bias);
                    // one ex2 per pixel
                    const float2 w = make_float2(ex2f(x.x), ex2f(x.y));
                    // numerator and weight sum: two two-lane FMA
                    num[c] = __ffma2_rn(w, g, num[c]);
                    den[c] = __ffma2_rn(w, f, den[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < P; ++c) sink += num[c].x + num[c].y + den[c].x + den[c].y;
    }
    out[tid] = sink;
}

// Counted units of one thread's loop iteration: thread-instructions of the measured kind, or taps
// for the mixed loop (a tap = one output pixel at one window offset).
double units_per_iteration(int op) {
    switch (op) {
    case OP_FFMA:
    case OP_FFMA2:
    case OP_EX2:
    case OP_EX2_H2:
    case OP_RED_SHARED:
    case OP_DP4A:
    case OP_HFMA2: return (double)kUnroll * kChains;
    case OP_TAP_FP16: return (double)kUnroll * (kChains / 2) * 2;   // two taps per pair
    case OP_TAP_PAIRED: return (double)kUnroll * (kChains / 2) * 2;   // two taps per pair
    default: return 0.0;
    }
}

cudaError_t launch(int op, int blocks, int iters, float *out, cudaStream_t st) {
    switch (op) {
    case OP_FFMA: rate_kernel<OP_FFMA><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_FFMA2: rate_kernel<OP_FFMA2><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_EX2: rate_kernel<OP_EX2><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_EX2_H2: rate_kernel<OP_EX2_H2><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_TAP_PAIRED: rate_kernel<OP_TAP_PAIRED><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_RED_SHARED: rate_kernel<OP_RED_SHARED><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_HFMA2: rate_kernel<OP_HFMA2><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_TAP_FP16: rate_kernel<OP_TAP_FP16><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    case OP_DP4A: rate_kernel<OP_DP4A><<<blocks, kThreads, 0, st>>>(out, iters, 1.0f); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

// Time `reps` launches of operation `op` (after one warm-up launch) on the current device with
// `blocks_per_sm` blocks of 256 threads per SM and `iters` loop iterations per thread.
// Writes the summed kernel time (CUDA events, milliseconds), the number of counted units
// (thread-instructions, or taps for the mixed loop) over those launches and the SM count.
// Returns 0, or the CUDA error code. Allocates its output buffer for the call and frees it.
extern "C" __attribute__((visibility("default"))) int alu_peak_run(int op, int blocks_per_sm, int iters, int reps,
                                                                  double *ms_out, double *units_out, int *sms_out) {
    if (op < 0 || op >= OP_COUNT || blocks_per_sm < 1 || iters < 1 || reps < 1 || !ms_out || !units_out || !sms_out)
        return (int)cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int blocks = sms * blocks_per_sm;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    if ((e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float))) != cudaSuccess) return (int)e;
    float ms = 0.0f;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess &&
        (e = launch(op, blocks, iters, out, st)) == cudaSuccess && (e = cudaEventRecord(e0, st)) == cudaSuccess) {
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch(op, blocks, iters, out, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    *ms_out = ms;
    *units_out = units_per_iteration(op) * iters * (double)blocks * kThreads * reps;
    *sms_out = sms;
    return 0;
}
