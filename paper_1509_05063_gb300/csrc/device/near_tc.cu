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
// done with N = 4R columns: the K range is doubled, [A | A_lo] against
// [[B_hi, B_lo]; [B_hi, 0]], and the two column halves are added in the
// epilogue.  The four K steps of a chunk accumulate into four separate
// tensor-memory accumulators, so that consecutive MMAs do not wait on one
// another's result; the epilogue sums them.
//
// Pipeline (warp-specialised: 128 producer threads, thread t = row t of the
// tile, plus one MMA warp; chunks of 8 complex columns): every producer keeps
// the next kTcAhead chunks of its row (and one input value u_j[column]) in
// flight in registers; for chunk c it waits until the MMAs of chunk
// c - kTcStages have released the stage, writes the raw weights and their lo
// parts into the stage in the canonical K-major no-swizzle layout (8-row x
// 16-byte core matrices; LBO = 128 B between K-adjacent core matrices,
// SBO = 1024 B between row groups), builds its B entries from the input
// values and arrives on the stage's "full" mbarrier.  Lane 0 of the MMA warp
// waits for "full", issues the chunk's four tcgen05.mma (M = 128, N = 4R,
// K = 8) and commits them to the stage's "empty" mbarrier.  No block barrier
// inside the loop.  The accumulators live in tensor memory and are read back
// with tcgen05.ld; the epilogue adds the CSR remainder and the local expansion
// Phi_q . gamma_c and writes out_q = u_q + kappa^2 (near + far).
// Every wait is bounded: on time-out a thread leaves its loop and flags the
// block, which then sets *err, lets its MMAs in flight finish (bounded), frees
// its tensor memory and leaves its rows unwritten.
#include <cstdint>

#include "device/cplx.cuh"
#include "device/kernels.cuh"

namespace lsd {
namespace {

constexpr int kTcRows = 128;          // rows per tile = MMA M = producer threads
constexpr int kTcThreads = kTcRows + 32;   // + one warp whose lane 0 issues the MMAs
constexpr int kTcKC = 8;              // complex columns per chunk
constexpr int kTcStages = 3;          // shared-memory stages (operand tiles of the MMAs in flight)
constexpr int kTcAhead = 4;           // chunks held in registers ahead of the one being prepared
constexpr int kTcKgroups = 2 * kTcKC / 2;  // 16-byte core-matrix columns per row: 4 raw + 4 lo
constexpr int kTcSBO = kTcKgroups * 128;   // bytes between 8-row groups (A and B)

__device__ __forceinline__ uint32_t s_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t s_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// x - (x with the 13 low mantissa bits cleared): exact in FP32
__device__ __forceinline__ float lo_tf32(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// poll an mbarrier phase at most `limit` times
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
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
  static constexpr int kStage = kA + kB;
  // independent accumulators (MMA chains): the four K steps of a chunk, times
  // two sets used by alternate chunks where tensor memory allows
  static constexpr int kSets = R >= 16 ? 1 : 2;
  static constexpr int kAcc = 4 * kSets;
  static constexpr int kTmemCols = kAcc * NN < 32 ? 32 : kAcc * NN;  // power of two >= 32
  // at most 512 / kTmemCols blocks may share an SM's tensor memory: pad the
  // shared memory so that no more blocks fit
  static constexpr int kBlocksMax = 512 / kTmemCols;
  static constexpr int kRaw = kTcStages * kStage + 128;            // + mbarriers, tensor-memory address, flag
  static constexpr int kFloor = 232448 / (kBlocksMax + 1) + 1;     // 227 KB / (max + 1)
  static constexpr int kBytes = kRaw > kFloor ? kRaw : kFloor;
};

// write (v.x, v.y) at B[n][kq], B[n][kq + 1] (kq even)
__device__ __forceinline__ void put_b(unsigned char* B, int n, int kq, float2 v) {
  *reinterpret_cast<float2*>(B + (n >> 3) * kTcSBO + (kq >> 2) * 128 + (n & 7) * 16 + (kq & 3) * 4) = v;
}

template <int R>
__global__ void __launch_bounds__(kTcThreads) k_near_tc(const int2* __restrict__ items,
                                                        const int64_t* __restrict__ occ_start,
                                                        const int64_t* __restrict__ blk_off,
                                                        const int* __restrict__ blk_seg,
                                                        const float2* __restrict__ Wb,
                                                        const int64_t* __restrict__ rem_row,
                                                        const int* __restrict__ rem_col,
                                                        const float2* __restrict__ rem_val,
                                                        const float2* __restrict__ u, int64_t N,
                                                        const float2* __restrict__ Phi,
                                                        const float2* __restrict__ gamma, int nocc, int nfb2,
                                                        float kappa2, float2* __restrict__ out,
                                                        int* __restrict__ err, int spin) {
  using Lay = TcLayout<R>;
  constexpr int NN = Lay::NN;
  static_assert(R * kTcKC <= kTcRows, "one input value per thread and chunk");
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kTcStages * Lay::kStage);     // stage written (128 arrivals)
  uint64_t* empty = full + kTcStages;                                             // stage read by the MMAs
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kTcStages * Lay::kStage + 64);
  int* sflag = reinterpret_cast<int*>(sm + kTcStages * Lay::kStage + 72);

  const int t = threadIdx.x, warp = t >> 5;
  const bool producer = t < kTcRows;
  const int2 item = items[blockIdx.x];
  const int k = item.x;
  const int* sg = blk_seg + 6 * k;
  const int l0 = sg[1], l1 = sg[3], l2 = sg[5];
  const int p0 = (l0 + 1) & ~1, p1 = (l1 + 1) & ~1;
  const int nblk = p0 + p1 + ((l2 + 1) & ~1);
  const int64_t r0 = occ_start[k];
  const int nrow = int(occ_start[k + 1] - r0);
  const int row = item.y + t;
  const bool valid = producer && row < nrow;
  const float2* wrow = Wb + blk_off[k] + int64_t(valid ? row : item.y) * nblk;
  const int nchunk = (nblk + kTcKC - 1) / kTcKC;
  // input value of this thread: RHS j, column cc of every chunk
  const int uj = t % R, ucc = t / R;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(s_u32(tslot)), "r"(Lay::kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(s_u32(&full[s])), "r"(kTcRows) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(s_u32(&empty[s])), "r"(1) : "memory");
    }
    *sflag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (producer) {
    // chunk c of this thread: its row's 8 complex weights (4 x 16 B) and, for
    // the first R * kTcKC threads, one input value u_j[column]; zero outside
    auto load = [&](int c, float4 (&w)[kTcKC / 2], float2& uv) {
      const int c0 = c * kTcKC;
#pragma unroll
      for (int p = 0; p < kTcKC / 2; ++p) {
        const int col = c0 + 2 * p;
        w[p] = (valid && col < nblk) ? __ldcs(reinterpret_cast<const float4*>(wrow + col))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      uv = make_float2(0.f, 0.f);
      if (t < R * kTcKC) {
        const int col = c0 + ucc;
        int64_t node = -1;
        if (col < p0) { if (col < l0) node = sg[0] + col; }
        else if (col < p0 + p1) { const int o = col - p0; if (o < l1) node = sg[2] + o; }
        else if (col < nblk) { const int o = col - p0 - p1; if (o < l2) node = sg[4] + o; }
        if (node >= 0) uv = u[int64_t(uj) * N + node];
      }
    };
    // register ring of the next kTcAhead chunks (loads in flight while earlier chunks are written)
    float4 wbuf[kTcAhead][kTcKC / 2];
    float2 ubuf[kTcAhead];
#pragma unroll
    for (int q = 0; q < kTcAhead; ++q)
      if (q < nchunk) load(q, wbuf[q], ubuf[q]);
    bool live = true;
    for (int cb = 0; cb < nchunk && live; cb += kTcAhead) {
#pragma unroll
      for (int q = 0; q < kTcAhead; ++q) {
        const int c = cb + q;
        if (c >= nchunk) break;
        const int s = c % kTcStages;
        // stage s was last read by the MMAs of chunk c - kTcStages
        if (c >= kTcStages && !mbar_wait(s_u32(&empty[s]), ((c - kTcStages) / kTcStages) & 1, spin)) {
          *sflag = 1;
          live = false;
          break;
        }
        unsigned char* A = sm + s * Lay::kStage;
        unsigned char* B = A + Lay::kA;
        // raw weights -> k-groups 0..3 of row t, their lo parts -> k-groups 4..7
#pragma unroll
        for (int p = 0; p < kTcKC / 2; ++p) {
          const float4 x = wbuf[q][p];
          *reinterpret_cast<float4*>(A + (t >> 3) * kTcSBO + p * 128 + (t & 7) * 16) = x;
          *reinterpret_cast<float4*>(A + (t >> 3) * kTcSBO + (4 + p) * 128 + (t & 7) * 16) =
              make_float4(lo_tf32(x.x), lo_tf32(x.y), lo_tf32(x.z), lo_tf32(x.w));
        }
        // B rows of chunk c: thread (cc, j) for complex column cc and RHS j
        if (t < R * kTcKC) {
          const float ur = ubuf[q].x, ui = ubuf[q].y;
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
        if (c + kTcAhead < nchunk) load(c + kTcAhead, wbuf[q], ubuf[q]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(s_u32(&full[s])) : "memory");
      }
    }
    // the last MMAs
    if (live && nchunk > 0 &&
        !mbar_wait(s_u32(&empty[(nchunk - 1) % kTcStages]), ((nchunk - 1) / kTcStages) & 1, spin))
      *sflag = 1;
  } else {
    // MMA warp (converged; lane 0 issues): four MMAs per chunk once its stage
    // is written, into four accumulators (M = 128, N = NN, A and B TF32
    // K-major, D FP32)
    const bool leader = (t & 31) == 0;
    const uint32_t idesc =
        (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NN >> 3) << 17) | (uint32_t(kTcRows >> 4) << 24);
    for (int c = 0; c < nchunk; ++c) {
      const int s = c % kTcStages;
      const bool ready = mbar_wait(s_u32(&full[s]), (c / kTcStages) & 1, spin);
      if (!__all_sync(0xffffffffu, ready)) {
        *sflag = 1;
        break;
      }
      if (leader) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = s_u32(sm + s * Lay::kStage), b0 = a0 + Lay::kA;
#pragma unroll
        for (int i = 0; i < 4; ++i) {      // K = 8 per MMA: k-groups 2i, 2i + 1
          const uint64_t da = s_desc(a0 + 2 * i * 128, 128, kTcSBO);
          const uint64_t db = s_desc(b0 + 2 * i * 128, 128, kTcSBO);
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                       :: "r"(tmem + uint32_t(((c % Lay::kSets) * 4 + i) * NN)), "l"(da), "l"(db), "r"(idesc),
                          "r"(c >= Lay::kSets ? 1 : 0)
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(s_u32(&empty[s])) : "memory");
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = *sflag == 0;
  if (ok && producer) {
    float d[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) d[i] = 0.f;
    if (nchunk > 0) {
#pragma unroll 1
      for (int a = 0; a < (nchunk < Lay::kSets ? 4 * nchunk : Lay::kAcc); ++a)   // sum of the accumulators used
#pragma unroll
        for (int q = 0; q < NN / 16; ++q) {
          float v[16];
          tmem_load16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(a * NN + 16 * q), v);
#pragma unroll
          for (int i = 0; i < 16; ++i) d[16 * q + i] += v[i];
        }
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
  } else if (!ok && t == 0) {
    atomicExch(err, 1);
    // let MMAs still in flight finish (bounded) before the tensor memory is released
    for (int s = 0; s < kTcStages; ++s) {
      mbar_wait(s_u32(&empty[s]), 0, spin);
      mbar_wait(s_u32(&empty[s]), 1, spin);
    }
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
  static unsigned long long attr = 0;
  if (first_on_device(attr)) {
    cudaError_t e = cudaFuncSetAttribute(k_near_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kBytes);
    if (e != cudaSuccess) return e;
  }
  if (d.n_items128 == 0) return cudaSuccess;
  k_near_tc<R><<<d.n_items128, kTcThreads, Lay::kBytes, st>>>(d.items128, d.occ_start, d.blk_off, d.blk_seg, d.Wb,
                                                           d.rem_row, d.rem_col, d.rem_val, u, d.N, d.Phi, d.gamma,
                                                           d.nocc, d.nfb2, float(d.kappa2), out, d.tc_err,
                                                              d.tc_spin);
  return cudaGetLastError();
}

template cudaError_t near_eval_tc<8>(const ApplyData<float2>&, const float2*, float2*, cudaStream_t);
template cudaError_t near_eval_tc<16>(const ApplyData<float2>&, const float2*, float2*, cudaStream_t);

}  // namespace lsd
