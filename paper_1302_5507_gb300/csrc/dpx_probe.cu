// Throughput probe of the integer operations the DP cell update uses.
//
// Each thread runs kChains independent dependency chains of one operation, so
// the measurement is bound by the issue rate of that operation's pipe, not by
// its latency.  The host entry times `iters` rounds with CUDA events and
// returns lane-operations per SM per clock (ops / (time x SMs x clock)), the
// number the ALU roofline of the score pass is built from.  Used by bench.py;
// not part of the alignment interface.
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

// max of two fp16x2 values held as bit patterns
__device__ __forceinline__ uint32_t hmax2_bits(uint32_t a, uint32_t b) {
    __half2 ha = *reinterpret_cast<__half2*>(&a), hb = *reinterpret_cast<__half2*>(&b);
    __half2 r = __hmax2(ha, hb);
    return *reinterpret_cast<uint32_t*>(&r);
}

enum Op {
    kViaddmaxS32 = 0, kVimax3S32 = 1, kVimax3ReluS32 = 2, kIaddS32 = 3, kImaxS32 = 4, kImadS32 = 5,
    kViaddmaxS16x2 = 6, kVimax3S16x2 = 7, kPrmt = 8,
    kVmaxS8x4 = 9, kVaddS8x4 = 10,                 // 4-way byte SIMD (signed max, saturating add)
    // half the chains one operation, half another: whether the two issue side by side
    kMixAddmaxImad = 11,                           // __viaddmax_s16x2 (ALU pipe) + IMAD (FMA pipe)
    kMixAddmaxPrmt = 12,                           // __viaddmax_s16x2 + PRMT (both ALU pipe)
    kLop3 = 13, kIadd3 = 14, kFfma = 15, kHmax2 = 16,   // alone: 3-input logic, 3-input add, fp32 FMA, fp16x2 max
    kMixAddmaxLop3 = 17, kMixAddmaxIadd3 = 18, kMixAddmaxFfma = 19, kMixAddmaxHmax2 = 20,
    kMixAddmaxShf = 21,                            // __viaddmax_s16x2 + funnel shift
    kNumOps = 22
};

template <int OP>
__global__ void __launch_bounds__(256) k_probe(int iters, uint32_t seed, uint32_t* sink) {
    uint32_t x[kChains], y = seed ^ threadIdx.x, z = seed * 3u + 7u;
    float xf[kChains];
    const float af = 1.0f + 1e-7f * (float)(seed & 7u), bf = 1e-3f * (float)threadIdx.x;
    const uint32_t one = blockDim.x >> 8;          // 1 at run time
#pragma unroll
    for (int c = 0; c < kChains; c++) { x[c] = seed + c * 977u + threadIdx.x; xf[c] = (float)x[c]; }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int rep = 0; rep < 16; rep++) {
#pragma unroll
            for (int c = 0; c < kChains; c++) {
                if (OP == kViaddmaxS32) x[c] = (uint32_t)__viaddmax_s32((int)x[c], (int)y, (int)z);
                if (OP == kVimax3S32) x[c] = (uint32_t)__vimax3_s32((int)x[c], (int)y, (int)(z + c));
                if (OP == kVimax3ReluS32) x[c] = (uint32_t)__vimax3_s32_relu((int)x[c], (int)y, (int)(z + c));
                if (OP == kIaddS32) x[c] = x[c] + y;
                if (OP == kImaxS32) x[c] = (uint32_t)max((int)x[c], (int)(y + c));
                if (OP == kImadS32) x[c] = x[c] * one + y;
                if (OP == kViaddmaxS16x2) x[c] = __viaddmax_s16x2(x[c], y, z);
                if (OP == kVimax3S16x2) x[c] = __vimax3_s16x2(x[c], y, z + c);
                if (OP == kPrmt) x[c] = __byte_perm(x[c], y, 0x5410 + c);
                if (OP == kVmaxS8x4) x[c] = __vmaxs4(x[c], y + c);
                if (OP == kVaddS8x4) x[c] = __vaddss4(x[c], y);
                if (OP == kMixAddmaxImad)
                    x[c] = (c & 1) ? x[c] * one + y : __viaddmax_s16x2(x[c], y, z);
                if (OP == kMixAddmaxPrmt)
                    x[c] = (c & 1) ? __byte_perm(x[c], y, 0x5410 + c) : __viaddmax_s16x2(x[c], y, z);
                if (OP == kLop3) x[c] = (x[c] & y) ^ (z | ~x[c]);
                if (OP == kIadd3) x[c] = x[c] + x[(c + 1) % kChains] + y;
                if (OP == kFfma) xf[c] = fmaf(xf[c], af, bf);
                if (OP == kHmax2) x[c] = hmax2_bits(x[c], x[(c + 1) % kChains]);
                if (OP == kMixAddmaxLop3)
                    x[c] = (c & 1) ? ((x[c] & y) ^ (z | ~x[c])) : __viaddmax_s16x2(x[c], y, z);
                if (OP == kMixAddmaxIadd3) x[c] = (c & 1) ? x[c] + x[(c + 1) % kChains] + y : __viaddmax_s16x2(x[c], y, z);
                if (OP == kMixAddmaxFfma) {
                    if (c & 1) xf[c] = fmaf(xf[c], af, bf);
                    else x[c] = __viaddmax_s16x2(x[c], y, z);
                }
                if (OP == kMixAddmaxHmax2) x[c] = (c & 1) ? hmax2_bits(x[c], x[(c + 1) % kChains]) : __viaddmax_s16x2(x[c], y, z);
                if (OP == kMixAddmaxShf)
                    x[c] = (c & 1) ? __funnelshift_l(x[c], y, (z + c) & 31u) : __viaddmax_s16x2(x[c], y, z);
            }
            y += 1;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= x[c] ^ __float_as_uint(xf[c]);
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = acc;     // keeps the chains alive
}

template <int OP>
float run(int blocks, int iters, uint32_t* sink) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_probe<OP><<<blocks, 256>>>(2, 1u, sink);           // warm-up
    cudaEventRecord(a);
    k_probe<OP><<<blocks, 256>>>(iters, 1u, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

// Lane-operations per SM per clock of operation `op` (see Op), measured at the
// given SM clock (MHz, as sampled by the caller); -1 on error.
extern "C" double sa_probe_ops_per_sm_clk(int op, double sm_mhz) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(uint32_t)) != cudaSuccess) return -1.0;
    const int blocks = sms * 8, iters = 2048;
    float ms = -1.f;
    switch (op) {
    case kViaddmaxS32: ms = run<kViaddmaxS32>(blocks, iters, sink); break;
    case kVimax3S32: ms = run<kVimax3S32>(blocks, iters, sink); break;
    case kVimax3ReluS32: ms = run<kVimax3ReluS32>(blocks, iters, sink); break;
    case kIaddS32: ms = run<kIaddS32>(blocks, iters, sink); break;
    case kImaxS32: ms = run<kImaxS32>(blocks, iters, sink); break;
    case kImadS32: ms = run<kImadS32>(blocks, iters, sink); break;
    case kViaddmaxS16x2: ms = run<kViaddmaxS16x2>(blocks, iters, sink); break;
    case kVimax3S16x2: ms = run<kVimax3S16x2>(blocks, iters, sink); break;
    case kPrmt: ms = run<kPrmt>(blocks, iters, sink); break;
    case kVmaxS8x4: ms = run<kVmaxS8x4>(blocks, iters, sink); break;
    case kVaddS8x4: ms = run<kVaddS8x4>(blocks, iters, sink); break;
    case kMixAddmaxImad: ms = run<kMixAddmaxImad>(blocks, iters, sink); break;
    case kMixAddmaxPrmt: ms = run<kMixAddmaxPrmt>(blocks, iters, sink); break;
    case kLop3: ms = run<kLop3>(blocks, iters, sink); break;
    case kIadd3: ms = run<kIadd3>(blocks, iters, sink); break;
    case kFfma: ms = run<kFfma>(blocks, iters, sink); break;
    case kHmax2: ms = run<kHmax2>(blocks, iters, sink); break;
    case kMixAddmaxLop3: ms = run<kMixAddmaxLop3>(blocks, iters, sink); break;
    case kMixAddmaxIadd3: ms = run<kMixAddmaxIadd3>(blocks, iters, sink); break;
    case kMixAddmaxFfma: ms = run<kMixAddmaxFfma>(blocks, iters, sink); break;
    case kMixAddmaxHmax2: ms = run<kMixAddmaxHmax2>(blocks, iters, sink); break;
    case kMixAddmaxShf: ms = run<kMixAddmaxShf>(blocks, iters, sink); break;
    default: break;
    }
    cudaFree(sink);
    if (ms <= 0.f || cudaGetLastError() != cudaSuccess) return -1.0;
    const double ops = (double)blocks * 256 * iters * 16 * kChains;
    return ops / ((double)ms * 1e-3) / sms / (sm_mhz * 1e6);
}

extern "C" int sa_probe_num_ops(void) { return kNumOps; }
