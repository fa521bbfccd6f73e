// k_diag.cu -- measurement of the GPU the library runs on: the sustained
// per-SM rates of the instruction kinds the raster kernels are built from
// (sdgr_pipe_rates), the denominators of their arithmetic roofline.
#include "sdgr_internal.cuh"

namespace sdgr {

// Diagnostic: sustained per-SM rate of one instruction kind, the denominators
// of the raster kernels' roofline.  Every thread runs eight independent
// chains of iters x 8 dependent instructions between two reads of the SM's
// cycle counter; the instructions are volatile asm, so none moves across the
// counter reads.  OP 0: fma.rn.f32; 1: ex2.approx.ftz.f32; 2:
// rcp.approx.ftz.f32, each followed by an fma (rcp of rcp is the identity,
// which the assembler may fold away; only the rcp are counted); 3: one ex2
// and seven fma per eight; 4: one rcp (with its fma) and seven fma per
// nine (what an SFU instruction costs inside an FP32 stream: one issue slot
// if the pipes overlap perfectly, more otherwise); 5: fma.rn.f32x2 (two FMAs
// per instruction); 6: fma.rn.f32 and lop3.b32 alternating; 7: fma.rn.f32x2
// and lop3.b32 alternating (how much FP32 work an issue slot carries beside
// integer work, one FMA or two).
__device__ __forceinline__ float probe_fma(float a) {
    float y;
    asm volatile("fma.rn.f32 %0, %1, 0f3F7FBE77, 0f3A03126F;" : "=f"(y) : "f"(a));  // a * 0.999 + 0.0005
    return y;
}
__device__ __forceinline__ float probe_ex2(float a) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-a));
    return y;
}
__device__ __forceinline__ float probe_rcp(float a) {
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}
__device__ __forceinline__ uint64_t probe_fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t y;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(y) : "l"(a), "l"(b), "l"(c));
    return y;
}
__device__ __forceinline__ uint32_t probe_lop3(uint32_t a) {
    uint32_t y;
    asm volatile("lop3.b32 %0, %1, 0x5a5a5a5a, 0x0f0f0f0f, 0x96;" : "=r"(y) : "r"(a));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(1024) k_pipe_rate(int iters, float *sink, unsigned long long *cycles) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.5f + 0.01f * (float)(threadIdx.x & 7) + 0.001f * (float)j;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (OP == 0 || (OP >= 3 && j >= 1)) a[j] = probe_fma(a[j]);
            else if (OP == 1 || OP == 3) a[j] = probe_ex2(a[j]);
            else a[j] = probe_fma(probe_rcp(a[j]));
        }
    }
    const long long t1 = clock64();
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == -1.f) sink[threadIdx.x] = s;  // never true: keeps the chains alive
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

// The packed and mixed kinds (5..7) in a kernel of their own, so that the
// code of the scalar kinds above stays as it was measured.
template <int OP>
__global__ void __launch_bounds__(1024) k_pipe_rate_pk(int iters, float *sink, unsigned long long *cycles) {
    float a[8];
    uint64_t p[8];
    uint32_t g[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        a[j] = 0.5f + 0.01f * (float)(threadIdx.x & 7) + 0.001f * (float)j;
        asm("mov.b64 %0, {%1, %2};" : "=l"(p[j]) : "f"(a[j]), "f"(a[j] + 0.1f));
        g[j] = threadIdx.x * 7u + (uint32_t)j;
    }
    uint64_t B2, C2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(B2) : "f"(0.999f));
    asm("mov.b64 %0, {%1, %1};" : "=l"(C2) : "f"(0.0005f));
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (OP == 5) {
                p[j] = probe_fma2(p[j], B2, C2);
            } else if (OP == 6) {
                a[j] = probe_fma(a[j]);
                g[j] = probe_lop3(g[j]);
            } else {
                p[j] = probe_fma2(p[j], B2, C2);
                g[j] = probe_lop3(g[j]);
            }
        }
    }
    const long long t1 = clock64();
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p[j]));
        s += a[j] + lo + hi + (float)g[j];
    }
    if (s == -1.f) sink[threadIdx.x] = s;  // never true: keeps the chains alive
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

cudaError_t launch_pipe_rate(int op, int iters, float *sink, unsigned long long *cycles, int *blocks_per_sm,
                             int sms, cudaStream_t s) {
    static void (*const kern[8])(int, float *, unsigned long long *) = {
        k_pipe_rate<0>, k_pipe_rate<1>, k_pipe_rate<2>, k_pipe_rate<3>,
        k_pipe_rate<4>, k_pipe_rate_pk<5>, k_pipe_rate_pk<6>, k_pipe_rate_pk<7>};
    if (op < 0 || op > 7) return cudaErrorInvalidValue;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern[op], 1024, 0);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    *blocks_per_sm = n;
    kern[op]<<<(unsigned)(sms * n), 1024, 0, s>>>(iters, sink, cycles);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr
