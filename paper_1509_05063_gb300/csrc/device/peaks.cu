// Throughput probes of this GPU's arithmetic units, for the roofline
// denominators of the kernels that are not HBM-bound: FP64 fused multiply-add
// on the CUDA cores, and TF32 MMA on the tensor cores (tcgen05; a reference
// rate beside the split-FP16 tensor-core near field).  Both run one launch
// over every SM and are timed with CUDA events on the launching stream.
#include <algorithm>
#include <cstdint>

#include "device/kernels.cuh"

namespace lsd {
namespace {

// kChains independent FMA chains per thread (enough to cover the FP64 pipe's
// latency), the loop body unrolled 4 times so that loop control is a small
// share of the issue slots; the result is stored so that nothing is optimised
// away
template <int kChains>
__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = double(threadIdx.x + c);
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1.2345) sink[blockIdx.x] = s;   // never true for the inputs used; keeps the chains live
}

__device__ __forceinline__ uint32_t s_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t s_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

constexpr int kMmaN = 256;          // M = 128, N = 256, K = 8 (TF32)
constexpr int kMmaBatch = 256;      // MMAs between commits

// one block per SM: lane 0 of warp 1 issues `iters` MMAs of 128 x 256 x 8
// (TF32 operands in shared memory, FP32 accumulator in tensor memory) into one
// accumulator, committing every kMmaBatch of them and waiting (bounded) for
// the commit before the next batch; *err is set if a wait gives up
__global__ void __launch_bounds__(64, 1) k_tf32_mma(int iters, int* err) {
  __shared__ __align__(1024) float A[128 * 8];
  __shared__ __align__(1024) float B[kMmaN * 8];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5;
  for (int i = t; i < 128 * 8; i += blockDim.x) A[i] = 1.0f / 1024;
  for (int i = t; i < kMmaN * 8; i += blockDim.x) B[i] = 1.0f / 1024;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(s_u32(&tslot)), "r"(kMmaN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (t == 32) {
    // K-major no-swizzle: 8-row groups 256 B apart (two 16-byte K columns of 8 rows)
    const uint64_t da = s_desc(s_u32(A), 128, 256), db = s_desc(s_u32(B), 128, 256);
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kMmaN >> 3) << 17) | (uint32_t(128 >> 4) << 24);
    uint32_t phase = 0;
    bool ok = true;
    for (int it = 0; it < iters && ok; ++it) {
      asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                   " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                   :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(it > 0 ? 1u : 0u) : "memory");
      if ((it + 1) % kMmaBatch == 0 || it + 1 == iters) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(s_u32(&bar)) : "memory");
        ok = false;
        for (int p = 0; p < (1 << 26) && !ok; ++p) {
          uint32_t done;
          asm volatile(
              "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
              : "=r"(done) : "r"(s_u32(&bar)), "r"(phase) : "memory");
          ok = done != 0;
        }
        phase ^= 1;
      }
    }
    if (!ok) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kMmaN) : "memory");
  }
}

}  // namespace

cudaError_t measure_peaks(double* fp64_tflops, double* tf32_tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  double* sink = nullptr;
  int* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * 64 * sms);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto timed = [&](auto launch, int reps) -> float {
    launch();                                         // warm-up
    cudaEventRecord(e0, 0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  if (e == cudaSuccess) {
    // the best of three shapes (chains per thread, resident blocks per SM)
    const int threads = 256, iters = 1 << 13;
    double best = 0;
    auto run = [&](auto kern, int chains, int per_sm) {
      const int blocks = per_sm * sms;
      const float ms = timed([&] { kern<<<blocks, threads>>>(iters, 0.999999, 1e-7, sink); }, 5);
      if (cudaGetLastError() != cudaSuccess) return false;
      best = std::max(best, 2.0 * chains * double(iters) * blocks * threads / (ms * 1e-3) / 1e12);
      return true;
    };
    if (!run(k_fp64_fma<8>, 8, 8) || !run(k_fp64_fma<16>, 16, 8) || !run(k_fp64_fma<32>, 32, 4))
      e = cudaErrorLaunchFailure;
    *fp64_tflops = best;
  }
  if (e == cudaSuccess) {
    const int iters = 1 << 16;
    const float ms = timed([&] { k_tf32_mma<<<sms, 64>>>(iters, err); }, 5);
    e = cudaGetLastError();
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    *tf32_tflops = flag ? -1.0 : 2.0 * 128 * kMmaN * 8 * double(iters) * sms / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (err) cudaFree(err);
  return e;
}

}  // namespace lsd
