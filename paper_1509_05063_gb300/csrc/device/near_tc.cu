// Near-field correction + evaluation + assembly for R complex64 right-hand
// sides on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Per work item = (occupied cell, 128 target rows) the near sum is one dense
// product  W_c (rows x nblk complex) . U (nblk x R complex)  against the cell's
// 3 x 3 neighbourhood (Eq. VolInt-Adj-NonAdj-I with the precomputed weights).
// It is written as one real GEMM with the weights as A, read from HBM exactly
// once in their stored layout (interleaved re, im along K):
//   A[m][2c] = Re W[m][c],  A[m][2c+1] = Im W[m][c]                (128 x 2 nblk)
//   B[2c][j] = Re u_j[c],   B[2c+1][j] = -Im u_j[c]      (j < R: real parts)
//   B[2c][R+j] = Im u_j[c], B[2c+1][R+j] = Re u_j[c]      (imaginary parts)
// so that D = A B holds Re(W u_j) in column j and Im(W u_j) in column R + j.
// FP32 accuracy from TF32 inputs (3xTF32): with x = hi(x) + lo(x), hi the TF32
// truncation (which is what the tensor core reads from an FP32 word) and lo
// exact in FP32,
//   D = A_hi B_hi + A_lo B_hi + A_hi B_lo  (the lo.lo term, 2^-22 relative, is dropped)
// done as ONE accumulator of N = 4R columns: the K range is doubled, [A | A_lo]
// against [[B_hi, B_lo]; [B_hi, 0]], and the two column halves are added in
// the epilogue.
//
// Pipeline (128 threads, thread t = row t of the tile; kTcStages shared-memory
// stages of 8 complex columns): cp.async streams the raw weights of chunk
// c + 2 into the canonical K-major no-swizzle layout (8-row x 16-byte core
// matrices; LBO = 128 B between K-adjacent core matrices, SBO = 1024 B between
// row groups) together with the chunk's input values u; for chunk c each
// thread writes the lo part of its own row and the B rows are built from the
// staged u; after one block barrier an elected thread issues the four
// tcgen05.mma (M = 128, N = 4R, K = 8) of the chunk and commits them to the
// stage's mbarrier, which every thread polls before it refills that stage.
// The accumulator lives in tensor memory and is read back with tcgen05.ld; the
// epilogue adds the CSR remainder and the local expansion Phi_q . gamma_c and
// writes out_q = u_q + kappa^2 (near + far).
// Every wait is bounded: on time-out the block sets *err, drains its copies,
// frees its tensor memory and leaves its rows unwritten.
#include <cstdint>

#include "device/cplx.cuh"
#include "device/kernels.cuh"

namespace lsd {
namespace {

constexpr int kTcRows = 128;          // rows per tile = MMA M
constexpr int kTcKC = 8;              // complex columns per chunk
constexpr int kTcStages = 4;
constexpr int kTcAhead = 2;           // chunks loaded ahead of the one being prepared
constexpr int kTcKgroups = 2 * kTcKC / 2;  // 16-byte core-matrix columns per row: 4 raw + 4 lo
constexpr int kTcSBO = kTcKgroups * 128;   // bytes between 8-row groups (A and B)
constexpr int kTcSpin = 1 << 22;      // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t s_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t s_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// x - (x with the 13 low mantissa bits cleared): exact in FP32
__device__ __forceinline__ float lo_tf32(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kTcSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_load16(uint32_t taddr, float* d) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) d[i] = __uint_as_float(r[i]);
}

template <int R>
struct TcLayout {
  static constexpr int NN = 4 * R;                                 // MMA N
  static constexpr int kA = kTcRows * kTcKgroups * 16;             // 16 KB: 128 rows x 32 fp32
  static constexpr int kB = NN * kTcKgroups * 16;                  // NN rows x 32 fp32
  static constexpr int kU = R * kTcKC * 8;                         // staged inputs of the chunk
  static constexpr int kStage = kA + kB + kU;
  static constexpr int kBytes = kTcStages * kStage + 128;          // + mbarriers, tensor-memory address, flag
  static constexpr int kTmemCols = NN < 32 ? 32 : NN;              // power of two >= 32
};

// write (v.x, v.y) at B[n][kq], B[n][kq + 1] (kq even)
__device__ __forceinline__ void put_b(unsigned char* B, int n, int kq, float2 v) {
  *reinterpret_cast<float2*>(B + (n >> 3) * kTcSBO + (kq >> 2) * 128 + (n & 7) * 16 + (kq & 3) * 4) = v;
}

template <int R>
__global__ void __launch_bounds__(kTcRows) k_near_tc(const int2* __restrict__ items,
                                                     const int64_t* __restrict__ occ_start,
                                                     const int64_t* __restrict__ blk_off,
                                                     const int* __restrict__ blk_seg, const float2* __restrict__ Wb,
                                                     const int64_t* __restrict__ rem_row,
                                                     const int* __restrict__ rem_col,
                                                     const float2* __restrict__ rem_val,
                                                     const float2* __restrict__ u, int64_t N,
                                                     const float2* __restrict__ Phi, const float2* __restrict__ gamma,
                                                     int nocc, int nfb2, float kappa2, float2* __restrict__ out,
                                                     int* __restrict__ err) {
  using Lay = TcLayout<R>;
  constexpr int NN = Lay::NN;
  static_assert(R * kTcKC <= kTcRows, "one staged input per thread");
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kTcStages * Lay::kStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kTcStages * Lay::kStage + 64);
  int* sflag = reinterpret_cast<int*>(sm + kTcStages * Lay::kStage + 96);

  const int t = threadIdx.x, warp = t >> 5;
  const int2 item = items[blockIdx.x];
  const int k = item.x;
  const int* sg = blk_seg + 6 * k;
  const int l0 = sg[1], l1 = sg[3], l2 = sg[5];
  const int p0 = (l0 + 1) & ~1, p1 = (l1 + 1) & ~1;
  const int nblk = p0 + p1 + ((l2 + 1) & ~1);
  const int64_t r0 = occ_start[k];
  const int nrow = int(occ_start[k + 1] - r0);
  const int row = item.y + t;
  const bool valid = row < nrow;
  const float2* wrow = Wb + blk_off[k] + int64_t(valid ? row : item.y) * nblk;
  const int nchunk = (nblk + kTcKC - 1) / kTcKC;
  // staged input of this thread: RHS j, column cc of every chunk
  const int uj = t % R, ucc = t / R;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(s_u32(tslot)), "r"(Lay::kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int s = 0; s < kTcStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(s_u32(&mbar[s])), "r"(1) : "memory");
    *sflag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  // raw weights of chunk c (k-groups 0..3 of row t) and its inputs -> stage c % kTcStages
  auto issue = [&](int c) {
    unsigned char* A = sm + (c % kTcStages) * Lay::kStage;
    const int c0 = c * kTcKC;
#pragma unroll
    for (int p = 0; p < kTcKC / 2; ++p) {
      const int col = c0 + 2 * p;
      const bool in = valid && col < nblk;
      const float2* src = wrow + (in ? col : 0);
      const uint32_t dst = s_u32(A + (t >> 3) * kTcSBO + p * 128 + (t & 7) * 16);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(in ? 16 : 0)
                   : "memory");
    }
    if (t < R * kTcKC) {
      const int col = c0 + ucc;
      int64_t node = -1;
      if (col < p0) { if (col < l0) node = sg[0] + col; }
      else if (col < p0 + p1) { const int o = col - p0; if (o < l1) node = sg[2] + o; }
      else if (col < nblk) { const int o = col - p0 - p1; if (o < l2) node = sg[4] + o; }
      const float2* src = node >= 0 ? u + int64_t(uj) * N + node : u;
      const uint32_t dst = s_u32(A + Lay::kA + Lay::kB + (ucc * R + uj) * 8);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(dst), "l"(src), "r"(node >= 0 ? 8 : 0)
                   : "memory");
    }
  };
  auto commit = [] { asm volatile("cp.async.commit_group;" ::: "memory"); };

  // M = 128, N = NN, A and B TF32 (K-major), D FP32
  const uint32_t idesc =
      (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NN >> 3) << 17) | (uint32_t(kTcRows >> 4) << 24);

  for (int c = 0; c < kTcAhead; ++c) {
    if (c < nchunk) issue(c);
    commit();
  }
  bool ok = true;
  int committed = 0;                       // chunks whose MMAs thread 0 has committed
  for (int c = 0; c < nchunk; ++c) {
    const int s = c % kTcStages;
    // refill stage (c + kTcAhead) % kTcStages, last read by the MMAs of chunk c + kTcAhead - kTcStages
    const int cl = c + kTcAhead - kTcStages;
    if (cl >= 0 && !mbar_wait(s_u32(&mbar[cl % kTcStages]), (cl / kTcStages) & 1)) *sflag = 1;
    if (c + kTcAhead < nchunk) issue(c + kTcAhead);
    commit();
    asm volatile("cp.async.wait_group %0;" :: "n"(kTcAhead) : "memory");
    unsigned char* A = sm + s * Lay::kStage;
    unsigned char* B = A + Lay::kA;
    // lo part of this thread's row -> k-groups 4..7
#pragma unroll
    for (int p = 0; p < kTcKC / 2; ++p) {
      const float4 x = *reinterpret_cast<const float4*>(A + (t >> 3) * kTcSBO + p * 128 + (t & 7) * 16);
      *reinterpret_cast<float4*>(A + (t >> 3) * kTcSBO + (4 + p) * 128 + (t & 7) * 16) =
          make_float4(lo_tf32(x.x), lo_tf32(x.y), lo_tf32(x.z), lo_tf32(x.w));
    }
    // B rows of chunk c: thread (cc, j) for complex column cc and RHS j (it staged that input itself)
    if (t < R * kTcKC) {
      const float2 v = *reinterpret_cast<const float2*>(A + Lay::kA + Lay::kB + (ucc * R + uj) * 8);
      const float ur = v.x, ui = v.y;
      const int j = uj, cc = ucc;
      put_b(B, j, 2 * cc, make_float2(ur, -ui));
      put_b(B, R + j, 2 * cc, make_float2(ui, ur));
      put_b(B, 2 * R + j, 2 * cc, make_float2(lo_tf32(ur), lo_tf32(-ui)));
      put_b(B, 3 * R + j, 2 * cc, make_float2(lo_tf32(ui), lo_tf32(ur)));
      put_b(B, j, 16 + 2 * cc, make_float2(ur, -ui));      // rows against A_lo: B_hi, then zero
      put_b(B, R + j, 16 + 2 * cc, make_float2(ui, ur));
      put_b(B, 2 * R + j, 16 + 2 * cc, make_float2(0.f, 0.f));
      put_b(B, 3 * R + j, 16 + 2 * cc, make_float2(0.f, 0.f));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (*sflag) { ok = false; break; }     // a wait above timed out (uniform after the barrier)
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = s_u32(A), b0 = s_u32(B);
#pragma unroll
      for (int i = 0; i < 4; ++i) {        // K = 8 per MMA: k-groups 2i, 2i + 1
        const uint64_t da = s_desc(a0 + 2 * i * 128, 128, kTcSBO);
        const uint64_t db = s_desc(b0 + 2 * i * 128, 128, kTcSBO);
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"((c > 0 || i > 0) ? 1 : 0) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(s_u32(&mbar[s])) : "memory");
      committed = c + 1;
    }
  }
  if (ok && nchunk > 0) {
    if (t == 0 && !mbar_wait(s_u32(&mbar[(nchunk - 1) % kTcStages]), ((nchunk - 1) / kTcStages) & 1)) *sflag = 1;
    __syncthreads();
    ok = !*sflag;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    float d[NN];
    if (nchunk > 0) {
#pragma unroll
      for (int q = 0; q < NN / 16; ++q) tmem_load16(tmem + (uint32_t(warp * 32) << 16) + 16 * q, d + 16 * q);
    } else {
#pragma unroll
      for (int i = 0; i < NN; ++i) d[i] = 0.f;
    }
    if (valid) {
      float2 acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = make_float2(d[j] + d[2 * R + j], d[R + j] + d[3 * R + j]);
      const int64_t q = r0 + row;
      for (int64_t e = rem_row[q]; e < rem_row[q + 1]; ++e) {
        const float2 w = rem_val[e];
        const int cidx = rem_col[e];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] = cfma(w, u[int64_t(j) * N + cidx], acc[j]);
      }
      const float2* ph = Phi + q * nfb2;
      for (int n = 0; n < nfb2; ++n) {
        const float2 p = ph[n];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] = cfma(p, gamma[(int64_t(j) * nocc + k) * nfb2 + n], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float2 uq = u[int64_t(j) * N + q];
        out[int64_t(j) * N + q] = make_float2(uq.x + kappa2 * acc[j].x, uq.y + kappa2 * acc[j].y);
      }
    }
  } else if (t == 0) {
    atomicExch(err, 1);
    // let the MMAs still in flight finish (bounded) before the tensor memory is released
    for (int c = committed > kTcStages ? committed - kTcStages : 0; c < committed; ++c)
      mbar_wait(s_u32(&mbar[c % kTcStages]), (c / kTcStages) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(Lay::kTmemCols)
                 : "memory");
}

}  // namespace

template <int R>
cudaError_t near_eval_tc(const ApplyData<float2>& d, const float2* u, float2* out, cudaStream_t st) {
  using Lay = TcLayout<R>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_near_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (d.n_items128 == 0) return cudaSuccess;
  k_near_tc<R><<<d.n_items128, kTcRows, Lay::kBytes, st>>>(d.items128, d.occ_start, d.blk_off, d.blk_seg, d.Wb,
                                                           d.rem_row, d.rem_col, d.rem_val, u, d.N, d.Phi, d.gamma,
                                                           d.nocc, d.nfb2, float(d.kappa2), out, d.tc_err);
  return cudaGetLastError();
}

template cudaError_t near_eval_tc<8>(const ApplyData<float2>&, const float2*, float2*, cudaStream_t);
template cudaError_t near_eval_tc<16>(const ApplyData<float2>&, const float2*, float2*, cudaStream_t);

}  // namespace lsd
