// Instruction-throughput probe for the arithmetic a Pauli-decomposition pass can
// use on this GPU: FP64 add (the paper's CMW sums of Eq. 4 in native double),
// FP32 add (the complex64 butterfly and its TwoSum compensation), 32/64-bit
// integer add, funnel shift and leading-zero count (the exact block-fixed-point
// butterfly), float<->double and int<->double conversions, and warp shuffles.
//
// Each kernel runs CHAINS independent dependency chains per thread over many
// warps, so the figure is issue throughput, not latency.  Results are printed
// as one JSON object per op: ops per clock per SM and ops per second, with the
// SM clock measured inside the kernel from %clock64 against %globaltimer.
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_alu probe_alu.cu
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CHAINS 8
#define ITERS 2048

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
  fprintf(stderr, "cuda error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); return 1; } } while (0)

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); return t;
}

// clk[0..1]: clock64 and globaltimer deltas measured by block 0, thread 0.
#define PROBE_PROLOGUE                                                        \
  uint64_t c0 = 0, g0 = 0;                                                    \
  if (blockIdx.x == 0 && threadIdx.x == 0) { g0 = gtimer(); c0 = clock64(); }
#define PROBE_EPILOGUE                                                        \
  if (blockIdx.x == 0 && threadIdx.x == 0) {                                  \
    uint64_t c1 = clock64(), g1 = gtimer();                                   \
    clk[0] = (double)(c1 - c0); clk[1] = (double)(g1 - g0); }

__global__ void k_dadd(double* out, double* clk, double b) {
  double a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(a[i]) : "d"(b));
  }
  PROBE_EPILOGUE
  double s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double* out, double* clk, double b) {
  double a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) asm volatile("fma.rn.f64 %0, %0, %1, %1;" : "+d"(a[i]) : "d"(b));
  }
  PROBE_EPILOGUE
  double s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_fadd(double* out, double* clk, float b) {
  float a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(a[i]) : "f"(b));
  }
  PROBE_EPILOGUE
  float s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_iadd32(double* out, double* clk, uint32_t b) {
  uint32_t a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
  }
  PROBE_EPILOGUE
  uint32_t s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_iadd64(double* out, double* clk, uint64_t b) {
  uint64_t a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) asm volatile("add.u64 %0, %0, %1;" : "+l"(a[i]) : "l"(b));
  }
  PROBE_EPILOGUE
  uint64_t s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

__global__ void k_shf(double* out, double* clk, uint32_t b) {
  uint32_t a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i)
      asm volatile("shf.l.wrap.b32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(b));
  }
  PROBE_EPILOGUE
  uint32_t s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_lop3(double* out, double* clk, uint32_t b) {
  uint32_t a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i)
      asm volatile("lop3.b32 %0, %0, %1, %1, 0x96;" : "+r"(a[i]) : "r"(b));
  }
  PROBE_EPILOGUE
  uint32_t s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// leading-zero count of a 64-bit word, folded back with an xor (2 ops / step)
__global__ void k_clz64(double* out, double* clk, uint64_t b) {
  uint64_t a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = (threadIdx.x + i) | (1ull << 40);
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
      uint32_t z;
      asm volatile("clz.b64 %0, %1;" : "=r"(z) : "l"(a[i]));
      asm volatile("xor.b32 %0, %0, %1;" : "+r"(z) : "r"((uint32_t)b));
      a[i] = (a[i] & ~0xFFull) | z;
    }
  }
  PROBE_EPILOGUE
  uint64_t s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

// double -> float -> double round trip (2 conversions / step)
__global__ void k_cvt_f64_f32(double* out, double* clk, double b) {
  double a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i + b;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
      float f;
      asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(a[i]));
      asm volatile("cvt.f64.f32 %0, %1;" : "=d"(a[i]) : "f"(f));
    }
  }
  PROBE_EPILOGUE
  double s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// double -> s64 -> double round trip (2 conversions / step)
__global__ void k_cvt_f64_s64(double* out, double* clk, double b) {
  double a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i + b;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
      long long l;
      asm volatile("cvt.rni.s64.f64 %0, %1;" : "=l"(l) : "d"(a[i]));
      asm volatile("cvt.rn.f64.s64 %0, %1;" : "=d"(a[i]) : "l"(l));
    }
  }
  PROBE_EPILOGUE
  double s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// reinterpret double bits as two 32-bit words and back (mov.b64 pack/unpack)
__global__ void k_movb64(double* out, double* clk, double b) {
  double a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i + b;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
      uint32_t lo, hi;
      asm volatile("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(a[i]));
      asm volatile("xor.b32 %0, %0, 1;" : "+r"(lo));
      asm volatile("mov.b64 %0, {%1, %2};" : "=d"(a[i]) : "r"(lo), "r"(hi));
    }
  }
  PROBE_EPILOGUE
  double s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_shfl(double* out, double* clk, uint32_t b) {
  uint32_t a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x + i + b;
  PROBE_PROLOGUE
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i)
      asm volatile("shfl.sync.bfly.b32 %0, %0, 1, 0x1f, 0xffffffff;" : "+r"(a[i]));
  }
  PROBE_EPILOGUE
  uint32_t s = 0; for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 16-byte vector copy, grid-stride (streaming HBM read + write)
__global__ void k_copy16(const double2* __restrict__ in, double2* __restrict__ out, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) out[i] = in[i];
}

typedef void (*kfn_d)(double*, double*, double);
typedef void (*kfn_f)(double*, double*, float);
typedef void (*kfn_u)(double*, double*, uint32_t);
typedef void (*kfn_l)(double*, double*, uint64_t);

struct Runner {
  double* out; double* clk; int blocks, threads, nsm;
  cudaEvent_t e0, e1;
  template <class F, class A>
  int run(const char* name, F f, A arg, double ops_per_step) {
    for (int w = 0; w < 2; ++w) f<<<blocks, threads>>>(out, clk, arg);
    CK(cudaGetLastError());
    CK(cudaEventRecord(e0));
    f<<<blocks, threads>>>(out, clk, arg);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0; CK(cudaEventElapsedTime(&ms, e0, e1));
    double hclk[2]; CK(cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost));
    double mhz = hclk[0] / hclk[1] * 1e3;
    double ops = (double)blocks * threads * ITERS * CHAINS * ops_per_step;
    double ops_s = ops / (ms * 1e-3);
    double per_clk_sm = ops_s / (nsm * mhz * 1e6);
    printf("{\"op\": \"%s\", \"ops_per_s\": %.4e, \"ops_per_clk_per_sm\": %.3f, \"sm_mhz\": %.0f, \"ms\": %.3f}\n",
           name, ops_s, per_clk_sm, mhz, ms);
    return 0;
  }
};

int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  printf("{\"gpu\": \"%s\", \"sms\": %d, \"cc\": \"%d.%d\"}\n", p.name, p.multiProcessorCount, p.major, p.minor);
  Runner r; r.nsm = p.multiProcessorCount; r.threads = 256; r.blocks = p.multiProcessorCount * 8;
  CK(cudaMalloc(&r.out, sizeof(double) * r.blocks * r.threads));
  CK(cudaMalloc(&r.clk, sizeof(double) * 2));
  CK(cudaEventCreate(&r.e0)); CK(cudaEventCreate(&r.e1));
  if (r.run("dadd", k_dadd, 1.0000001, 1.0)) return 1;
  if (r.run("dfma", k_dfma, 0.9999999, 1.0)) return 1;
  if (r.run("fadd", k_fadd, 1.0f, 1.0)) return 1;
  if (r.run("iadd32", k_iadd32, 3u, 1.0)) return 1;
  if (r.run("iadd64", k_iadd64, 3ull, 1.0)) return 1;
  if (r.run("shf", k_shf, 5u, 1.0)) return 1;
  if (r.run("lop3", k_lop3, 5u, 1.0)) return 1;
  if (r.run("clz64+xor+merge", k_clz64, 7ull, 1.0)) return 1;
  if (r.run("cvt_f64_f32_roundtrip(2cvt)", k_cvt_f64_f32, 0.5, 2.0)) return 1;
  if (r.run("cvt_f64_s64_roundtrip(2cvt)", k_cvt_f64_s64, 0.5, 2.0)) return 1;
  if (r.run("movb64_unpack_xor_pack", k_movb64, 0.5, 1.0)) return 1;
  if (r.run("shfl_bfly", k_shfl, 1u, 1.0)) return 1;
  {
    size_t n = (size_t)1 << 28;  // 4 GiB of 16-byte elements per buffer
    double2 *a = nullptr, *b = nullptr;
    CK(cudaMalloc(&a, n * 16)); CK(cudaMalloc(&b, n * 16));
    CK(cudaMemset(a, 0, n * 16));
    for (int bpsm = 2; bpsm <= 8; bpsm *= 2) {
      int blocks = p.multiProcessorCount * bpsm;
      float best = 1e30f;
      for (int rep = 0; rep < 6; ++rep) {
        CK(cudaEventRecord(r.e0));
        k_copy16<<<blocks, 512>>>(a, b, n);
        CK(cudaEventRecord(r.e1));
        CK(cudaEventSynchronize(r.e1));
        float ms; CK(cudaEventElapsedTime(&ms, r.e0, r.e1));
        if (rep > 0 && ms < best) best = ms;
      }
      printf("{\"op\": \"copy16\", \"blocks_per_sm\": %d, \"gbs\": %.1f, \"ms\": %.3f}\n",
             bpsm, 2.0 * n * 16 / (best * 1e-3) / 1e9, best);
    }
    CK(cudaFree(a)); CK(cudaFree(b));
  }
  return 0;
}
