// Near-field correction + evaluation + assembly for R complex64 right-hand
// sides on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Per work item = (occupied cell, up to 128 target rows) the near sum is one
// dense product  W_c (rows x nblk complex) . U (nblk x R complex)  against the
// cell's 3 x 3 neighbourhood (Eq. VolInt-Adj-NonAdj-I with the precomputed
// weights), written as one real GEMM with the weights as A (interleaved re, im
// along K):
//   A[m][2c] = Re W[m][c],  A[m][2c+1] = Im W[m][c]
//   B[2c][j] = Re u_j[c],   B[2c+1][j] = -Im u_j[c]      (columns j < R: real parts)
//   B[2c][R+j] = Im u_j[c], B[2c+1][R+j] = Re u_j[c]      (imaginary parts)
// so that D = A B holds Re(W u_j) in column j and Im(W u_j) in column R + j.
//
// Split FP16 operands (kind::f16, FP32 accumulation).  A row's weights are
// scaled by a power of two s_m that puts the row's largest magnitude in
// [2^14, 2^15) and split as x s_m = hi + lo with hi = fp16(x s_m) and
// lo = fp16(x s_m - hi), together 22 significant bits; right-hand side j is
// scaled by a power of two t_j the same way.  Then
//   D = A_hi B_hi + A_hi B_lo + A_lo B_hi    (the lo.lo term, 2^-22 relative, is dropped)
// as two MMAs per K step into one accumulator: A_hi against [B_hi | B_lo]
// (N = 4R columns) and A_lo against B_hi (N = 2R, accumulating into the first
// 2R columns); the epilogue adds the two column halves and divides by s_m t_j.
// An MMA instruction costs about the same time for N = 32 and N = 64 here, so
// the work per byte of weights is set by the instruction count: FP16 takes
// K = 16 per instruction where TF32 takes 8, which halves it, and the lo parts
// come from HBM with the hi parts (the same 4 bytes per real weight as FP32),
// so no thread touches the weight stream.
//
// Storage (built once at plan time from the row-major blocks): per work item
// and chunk of kKC complex columns, the hi parts of the item's rows in groups
// of 8 as the canonical K-major no-swizzle core-matrix layout (8 rows x 16
// bytes per core matrix, 128 bytes between K-adjacent core matrices, 512
// bytes between row groups), only the row groups that hold rows, then the lo
// parts in the same layout.  Two bulk copies (cp.async.bulk, completion
// counted on an mbarrier) move a chunk from HBM into a weight stage.
//
// Persistent, warp-specialised, one block per SM walking its own list of work
// items (lists balanced at plan time, longest first):
//   warp 0      lane 0 issues the bulk copies into a ring of kNA weight stages
//               (L2 evict-first: the weights are read once);
//   warp 1      lane 0 issues the MMAs and commits them to the release barriers;
//   warps 2..5  (128 threads) per item: read the accumulator from tensor memory
//               (two items in flight), add the CSR remainder and the local
//               expansion Phi_q . gamma_c and write out_q = u_q + kappa^2 (near + far);
//   warps 6..   one warp per operand slot: the B operand (scaled hi and lo) of
//               the chunks that use its slot, from the input vectors (gathers
//               issued one owned chunk ahead).
// Every wait is bounded by `spin` polls and also gives up once another role
// has flagged a failure; then the block sets *err, waits (with a fixed bound
// that does not depend on `spin`) for its own MMAs and bulk copies still in
// flight, frees its tensor memory and returns, leaving its rows unwritten.
#include <algorithm>
#include <cstdint>

#include <cuda_fp16.h>

#include "device/cplx.cuh"
#include "device/kernels.cuh"

namespace lsd {
namespace {

constexpr int kTcRows = 128;                 // rows per item = MMA M
constexpr int kKC = 16;                      // complex columns per chunk (K = 32 real)
constexpr int kKG = 2 * kKC / 8;             // 16-byte core-matrix columns per row (8 fp16 each): 4
constexpr int kRowGroup = 8 * kKG * 16;      // bytes of one 8-row group of a chunk (hi or lo): 512
constexpr int kHalf = 16 * kRowGroup;        // 128 rows, hi or lo: 8 KB
constexpr int kAStage = 2 * kHalf;           // a weight stage: hi, then lo
constexpr int kNA = 12;                      // weight stages (bulk-copy ring)
constexpr int kNC = 6;                       // B operand slots = B warps
constexpr int kAhead = 1;                    // owned chunks a B warp gathers ahead of its split (1 or 2)
constexpr int kSets = 2;                     // accumulator sets per item (K step k uses set k mod kSets)
constexpr int kThreads = 32 * (6 + kNC);
constexpr int kDrainPolls = 1 << 28;         // bound of the final waits on the block's own MMAs / copies

__device__ __forceinline__ uint32_t s_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t s_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// one poll of an mbarrier phase.  try_wait may suspend the thread for a while
// and, measured here, wakes it a few hundred cycles after the phase completes;
// test_wait returns at once.  The latency-critical roles (bulk copies, MMA
// issue, B operands) spin on test_wait; the epilogue, which waits a whole
// item's main loop, sleeps in try_wait and leaves the issue slots to them.
template <bool kSpin>
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  if constexpr (kSpin)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ int ld_flag(const int* f) {
  int v;
  asm volatile("ld.volatile.shared.b32 %0, [%1];" : "=r"(v) : "r"(s_u32(f)) : "memory");
  return v;
}

__device__ __forceinline__ void set_flag(int* f, int v) {
  asm volatile("st.volatile.shared.b32 [%0], %1;" :: "r"(s_u32(f)), "r"(v) : "memory");
}

// wait for a phase: at most `limit` polls, and give up as soon as the block's
// failure flag is set; on time-out the flag is set.  Every waiter below waits
// for the phases of its barrier in order: one that skipped a phase would see
// the earlier phase of the same parity as complete.
template <bool kSpin = true>
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, int limit, int* flag) {
  for (int it = 0; it < limit; ++it) {
    if (mbar_try<kSpin>(bar, parity)) return true;
    if (ld_flag(flag)) return false;
  }
  set_flag(flag, 1);
  return false;
}

// the same with a fixed bound and no flag (the block's own MMAs and copies,
// which depend on nothing else)
__device__ __forceinline__ bool drain_phase(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kDrainPolls; ++it)
    if (mbar_try<false>(bar, parity)) return true;
  return false;
}

// 16 consecutive accumulator columns of this thread's lane; the load and its
// wait are one asm statement, so no register is read before the data is there
__device__ __forceinline__ void tmem_load16(uint32_t taddr, float* d) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) d[i] = __uint_as_float(r[i]);
}

template <int R>
struct TcLayout {
  static constexpr int NN = 4 * R;                              // MMA N of [B_hi | B_lo]
  static constexpr int kB = NN * kKG * 16;                      // B operand of a chunk
  static constexpr int kTmemCols = 2 * kSets * NN < 32 ? 32 : 2 * kSets * NN;
  static constexpr int kBarOff = kNA * kAStage + kNC * kB;
  // + mbarriers (2 kNA + 2 kNC + 5), tensor-memory address, flag
  static constexpr int kBytes = kBarOff + 8 * (2 * kNA + 2 * kNC + 5) + 16;
};

// (hi, lo) fp16 split of a scaled value
__device__ __forceinline__ void split16(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// write the fp16 pair (v0, v1) at B[n][kq], B[n][kq + 1] (kq even)
__device__ __forceinline__ void put_b(unsigned char* B, int n, int kq, __half v0, __half v1) {
  *reinterpret_cast<__half2*>(B + (n >> 3) * kRowGroup + (kq >> 3) * 128 + (n & 7) * 16 + (kq & 7) * 2) =
      __halves2half2(v0, v1);
}

struct ItemGeom {
  int k, row0, nrow, nblk, nchunk, groups;
  int64_t off;   // byte offset / 8 of the item's first chunk in the tile layout
};

__device__ __forceinline__ ItemGeom item_geom(int it, const int2* items, const int64_t* tile_off,
                                              const int64_t* occ_start, const int* blk_seg) {
  const int2 item = items[it];
  ItemGeom g;
  g.k = item.x;
  g.row0 = item.y;
  const int* sg = blk_seg + 6 * g.k;
  g.nblk = ((sg[1] + 1) & ~1) + ((sg[3] + 1) & ~1) + ((sg[5] + 1) & ~1);
  g.nchunk = (g.nblk + kKC - 1) / kKC;
  const int rows = int(occ_start[g.k + 1] - occ_start[g.k]) - g.row0;
  g.nrow = rows < kTcRows ? rows : kTcRows;
  g.groups = (g.nrow + 7) >> 3;
  g.off = tile_off[it];
  return g;
}

// power-of-two scale that puts m (> 0, normal) in [2^14, 2^15): 2^(14 - floor(log2 m))
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m >= 1.17549435e-38f) || !(m < 3.0e38f)) return 1.f;
  const int e = int((__float_as_uint(m) >> 23) & 0xFF) - 127;   // floor(log2 m)
  return ldexpf(1.f, 14 - e < 126 ? 14 - e : 126);
}

// per right-hand side j (blockIdx.y): the largest |Re u_j[q]|, |Im u_j[q]|,
// as the bits of a non-negative float (whose order is the integers' order)
// maxed into tmax[j], which the caller zeroes first
constexpr int kScaleBlocks = 32;
__global__ void __launch_bounds__(256) k_rhs_max(const float2* __restrict__ u, int64_t N,
                                                 unsigned* __restrict__ tmax) {
  const float2* v = u + int64_t(blockIdx.y) * N;
  float m = 0.f;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < N; q += int64_t(gridDim.x) * blockDim.x)
    m = fmaxf(m, fmaxf(fabsf(v[q].x), fabsf(v[q].y)));
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) atomicMax(&tmax[blockIdx.y], __float_as_uint(m));
}

template <int R>
__global__ void __launch_bounds__(kThreads, 1) k_near_tc(const int2* __restrict__ items, const int* __restrict__ bptr,
                                                         const int* __restrict__ blist,
                                                         const int64_t* __restrict__ tile_off,
                                                         const int64_t* __restrict__ occ_start,
                                                         const int* __restrict__ blk_seg,
                                                         const unsigned char* __restrict__ Wt,
                                                         const float* __restrict__ rscale,
                                                         const unsigned* __restrict__ tmax,
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
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Aring = sm;                                  // kNA x (8 KB hi + 8 KB lo)
  unsigned char* Bring = sm + kNA * kAStage;                  // kNC x B operand
  uint64_t* a_full = reinterpret_cast<uint64_t*>(sm + Lay::kBarOff);
  uint64_t* a_empty = a_full + kNA;
  uint64_t* b_ready = a_empty + kNA;                          // B written (32 arrivals)
  uint64_t* b_empty = b_ready + kNC;                          // B read by the MMAs
  uint64_t* acc_full = b_empty + kNC;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  int* sflag = reinterpret_cast<int*>(tslot + 1);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int p_begin = bptr[blockIdx.x], p_end = bptr[blockIdx.x + 1];   // this block's items

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(s_u32(tslot)), "r"(Lay::kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 32) {
    for (int s = 0; s < kNA; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&a_full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&a_empty[s])) : "memory");
    }
    for (int s = 0; s < kNC; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" :: "r"(s_u32(&b_ready[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&b_empty[s])) : "memory");
    }
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&acc_full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" :: "r"(s_u32(&acc_empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(drain)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sflag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ------------------------------------------------ bulk copies of the weight chunks
    if (lane == 0) {
      // the weights are read once: first in line for L2 eviction, so that the
      // input vectors the B warps gather stay in L2 beside the stream
      uint64_t stream_pol;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_pol));
      int g = 0;   // chunk counter of this block
      bool live = true;
      for (int ip = p_begin; ip < p_end && live; ++ip) {
        const int it = blist[ip];
        const ItemGeom ig = item_geom(it, items, tile_off, occ_start, blk_seg);
        const uint32_t half_bytes = uint32_t(ig.groups) * kRowGroup;
        for (int c = 0; c < ig.nchunk; ++c, ++g) {
          const int s = g % kNA, use = g / kNA;
          if (use > 0 && !wait_phase(s_u32(&a_empty[s]), (use - 1) & 1, spin, sflag)) {
            live = false;
            break;
          }
          const unsigned char* src = Wt + 8 * ig.off + int64_t(c) * 2 * half_bytes;
          const uint32_t dst = s_u32(Aring + s * kAStage), bar = s_u32(&a_full[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(2 * half_bytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
              :: "r"(dst), "l"(src), "r"(half_bytes), "r"(bar), "l"(stream_pol) : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
              :: "r"(dst + kHalf), "l"(src + half_bytes), "r"(half_bytes), "r"(bar), "l"(stream_pol) : "memory");
        }
      }
      // every copy issued must have landed before the block leaves (shared
      // memory is written by them): wait for the last phase of each stage
      const int issued = g;
      for (int s = 0; s < kNA && s < issued; ++s) {
        const int last_use = (issued - 1 - s) / kNA;
        if (!drain_phase(s_u32(&a_full[s]), last_use & 1)) set_flag(sflag, 2);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      // kind::f16: D F32, A and B F16, both K-major
      const uint32_t idesc1 = (1u << 4) | (uint32_t(NN >> 3) << 17) | (uint32_t(kTcRows >> 4) << 24);
      const uint32_t idesc2 = (1u << 4) | (uint32_t((NN / 2) >> 3) << 17) | (uint32_t(kTcRows >> 4) << 24);
      int g = 0, tile = 0;
      bool live = true, issued = false;
      for (int ip = p_begin; ip < p_end && live; ++ip, ++tile) {
        const int it = blist[ip];
        const ItemGeom ig = item_geom(it, items, tile_off, occ_start, blk_seg);
        const int b = tile & 1, bu = tile >> 1;
        if (bu > 0 && !wait_phase(s_u32(&acc_empty[b]), (bu - 1) & 1, spin, sflag)) {
          live = false;
          break;
        }
        const uint32_t acc0 = tmem + uint32_t(kSets * b * NN);
        for (int c = 0; c < ig.nchunk; ++c, ++g) {
          const int sa = g % kNA, sb = g % kNC;
          if (!wait_phase(s_u32(&b_ready[sb]), (g / kNC) & 1, spin, sflag) ||
              !wait_phase(s_u32(&a_full[sa]), (g / kNA) & 1, spin, sflag)) {
            live = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = s_u32(Aring + sa * kAStage), b0 = s_u32(Bring + sb * Lay::kB);
#pragma unroll
          for (int i = 0; i < kKG / 2; ++i) {      // K = 16 per MMA: core-matrix columns 2i, 2i + 1
            const uint64_t dh = s_desc(a0 + 2 * i * 128, 128, kRowGroup);
            const uint64_t dl = s_desc(a0 + kHalf + 2 * i * 128, 128, kRowGroup);
            const uint64_t db = s_desc(b0 + 2 * i * 128, 128, kRowGroup);
            const int ks = c * (kKG / 2) + i;        // K step of the item: accumulator set ks mod kSets
            const uint32_t acc = acc0 + uint32_t((ks % kSets) * NN);
            const uint32_t accum = ks >= kSets ? 1u : 0u;
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         :: "r"(acc), "l"(dh), "l"(db), "r"(idesc1), "r"(accum) : "memory");
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         :: "r"(acc), "l"(dl), "l"(db), "r"(idesc2), "r"(1u) : "memory");
          }
          issued = true;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(s_u32(&a_empty[sa])) : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(s_u32(&b_empty[sb])) : "memory");
        }
        if (!live) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(s_u32(&acc_full[b])) : "memory");
      }
      // the tensor memory may only be released once every MMA of this block has
      // completed: one more commit tracks all of them
      if (issued) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(s_u32(drain)) : "memory");
        if (!drain_phase(s_u32(drain), 0)) set_flag(sflag, 2);
      }
    }
  } else if (warp >= 6) {
    // ------------------------------------------------ B operands (scaled hi and lo) from the input vectors
    // warp bw owns operand slot bw: it builds the B of chunks g = bw, bw + kNC,
    // ... of this block.  Value v = lane + 32 i of a chunk is (RHS j = v % R,
    // column cc = v / R).
    constexpr int kVals = R * kKC / 32;
    static_assert(R * kKC % 32 == 0 && 32 % R == 0, "B entries per lane; RHS j = lane mod R");
    const int bw = warp - 6;
    const int j = lane % R;                        // this lane's right-hand side, for every value it moves
    const float tsj = pow2_scale(__uint_as_float(tmax[j]));
    const float2* uj = u + int64_t(j) * N;
    // gathers of a chunk's inputs go out kAhead owned chunks ahead: the loads
    // of chunk g are in flight while chunks g - kNC, ... are split into the slot
    float2 pa[kVals], pb[kVals], nx[kVals];
    int ua = -1, ub = -1;                          // uses of the pending chunks (-1: none)
    auto build = [&](const float2* uv, int use) -> bool {
      if (use > 0 && !wait_phase(s_u32(&b_empty[bw]), (use - 1) & 1, spin, sflag)) return false;
      unsigned char* B = Bring + bw * Lay::kB;
#pragma unroll
      for (int i = 0; i < kVals; ++i) {
        const int cc = (lane + 32 * i) / R;
        const float ur = uv[i].x * tsj, ui = uv[i].y * tsj;
        __half rh, rl, ih, il, mh, ml;
        split16(ur, rh, rl);
        split16(ui, ih, il);
        split16(-ui, mh, ml);
        put_b(B, j, 2 * cc, rh, mh);             // real-part rows: (Re, -Im)
        put_b(B, R + j, 2 * cc, ih, rh);         // imaginary-part rows: (Im, Re)
        put_b(B, 2 * R + j, 2 * cc, rl, ml);
        put_b(B, 3 * R + j, 2 * cc, il, rl);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(s_u32(&b_ready[bw])) : "memory");
      return true;
    };
    int g = 0;
    bool live = true;
    for (int ip = p_begin; ip < p_end && live; ++ip) {
      const int it = blist[ip];
      const ItemGeom ig = item_geom(it, items, tile_off, occ_start, blk_seg);
      const int* sg = blk_seg + 6 * ig.k;
      const int l0 = sg[1], l1 = sg[3], l2 = sg[5];
      const int p0 = (l0 + 1) & ~1, p1 = (l1 + 1) & ~1;
      for (int c = 0; c < ig.nchunk; ++c, ++g) {
        if (g % kNC != bw) continue;
#pragma unroll
        for (int i = 0; i < kVals; ++i) {
          const int col = c * kKC + (lane + 32 * i) / R;
          int64_t node = -1;
          if (col < p0) { if (col < l0) node = sg[0] + col; }
          else if (col < p0 + p1) { const int o = col - p0; if (o < l1) node = sg[2] + o; }
          else if (col < ig.nblk) { const int o = col - p0 - p1; if (o < l2) node = sg[4] + o; }
          nx[i] = node >= 0 ? uj[node] : make_float2(0.f, 0.f);
        }
        if constexpr (kAhead == 1) {
          if (ua >= 0 && !build(pa, ua)) { live = false; break; }
#pragma unroll
          for (int i = 0; i < kVals; ++i) pa[i] = nx[i];
          ua = g / kNC;
        } else {
          if (ua >= 0 && !build(pa, ua)) { live = false; break; }
#pragma unroll
          for (int i = 0; i < kVals; ++i) { pa[i] = pb[i]; pb[i] = nx[i]; }
          ua = ub;
          ub = g / kNC;
        }
      }
    }
    if (live && ua >= 0) live = build(pa, ua);
    if constexpr (kAhead == 2)
      if (live && ub >= 0) build(pb, ub);
  } else {
    // ------------------------------------------------ epilogue (warps 2..5)
    const int row_in = 32 * (warp & 3) + lane;     // tensor-memory lane quarter of this warp
    float inv_t[R];
#pragma unroll
    for (int j = 0; j < R; ++j) inv_t[j] = 1.f / pow2_scale(__uint_as_float(tmax[j]));
    int tile = 0;
    for (int ip = p_begin; ip < p_end; ++ip, ++tile) {
      const int it = blist[ip];
      const ItemGeom ig = item_geom(it, items, tile_off, occ_start, blk_seg);
      const int b = tile & 1, bu = tile >> 1;
      float d[NN], d2[NN];
      // the warp's lanes decide together (tcgen05.ld is warp-collective)
      if (!__all_sync(0xffffffffu, wait_phase<false>(s_u32(&acc_full[b]), bu & 1, spin, sflag))) {
        set_flag(sflag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ig.nchunk > 0) {
        const uint32_t ta = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(kSets * b * NN);
#pragma unroll
        for (int q = 0; q < NN / 16; ++q) tmem_load16(ta + uint32_t(16 * q), d + 16 * q);
        const int used = ig.nchunk * (kKG / 2) < kSets ? ig.nchunk * (kKG / 2) : kSets;   // sets written
#pragma unroll
        for (int st = 1; st < kSets; ++st) {
          if (st >= used) break;
#pragma unroll
          for (int q = 0; q < NN / 16; ++q) tmem_load16(ta + uint32_t(st * NN + 16 * q), d2 + 16 * q);
#pragma unroll
          for (int i = 0; i < NN; ++i) d[i] += d2[i];
        }
      } else {
#pragma unroll
        for (int i = 0; i < NN; ++i) d[i] = 0.f;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(s_u32(&acc_empty[b])) : "memory");
      if (row_in < ig.nrow) {
        const int64_t q = occ_start[ig.k] + ig.row0 + row_in;
        const float rs = rscale[q];
        float2 acc[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const float f = rs * inv_t[j];
          acc[j] = make_float2((d[j] + d[2 * R + j]) * f, (d[R + j] + d[3 * R + j]) * f);
        }
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
          for (int j = 0; j < R; ++j) acc[j] = cfma(p, gamma[(int64_t(j) * nocc + ig.k) * nfb2 + n], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const float2 uq = u[int64_t(j) * N + q];
          out[int64_t(j) * N + q] = make_float2(uq.x + kappa2 * acc[j].x, uq.y + kappa2 * acc[j].y);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (t == 0 && *sflag != 0) atomicExch(err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(Lay::kTmemCols)
                 : "memory");
  }
}

// tile layout of the weights from the row-major blocks: block = work item.
// Row scales first (s_m puts the row's largest |Re|, |Im| in [2^14, 2^15);
// rscale[q] = 1 / s_m for the row's node q), then per chunk c and row group
// the hi parts, then the lo parts: fp16 element (row m, real index k of the
// chunk) at byte (c * 2 * groups + part * groups + m / 8) * 512 + (k / 8) * 128
// + (m % 8) * 16 + (k % 8) * 2 from the item's start; zero past the columns
__global__ void __launch_bounds__(256) k_tile_weights(const int2* __restrict__ items,
                                                      const int64_t* __restrict__ tile_off,
                                                      const int64_t* __restrict__ occ_start,
                                                      const int64_t* __restrict__ blk_off,
                                                      const int* __restrict__ blk_seg, const float2* __restrict__ Wb,
                                                      unsigned char* __restrict__ Wt, float* __restrict__ rscale) {
  __shared__ float srow[kTcRows];
  const ItemGeom ig = item_geom(blockIdx.x, items, tile_off, occ_start, blk_seg);
  const float2* src = Wb + blk_off[ig.k] + int64_t(ig.row0) * ig.nblk;
  for (int m = threadIdx.x; m < kTcRows; m += blockDim.x) {
    float mx = 0.f;
    if (m < ig.nrow)
      for (int c = 0; c < ig.nblk; ++c) {
        const float2 w = src[int64_t(m) * ig.nblk + c];
        mx = fmaxf(mx, fmaxf(fabsf(w.x), fabsf(w.y)));
      }
    const float s = pow2_scale(mx);
    srow[m] = s;
    if (m < ig.nrow) rscale[occ_start[ig.k] + ig.row0 + m] = 1.f / s;
  }
  __syncthreads();
  __half* dst = reinterpret_cast<__half*>(Wt + 8 * ig.off);
  const int64_t per_half = int64_t(ig.groups) * kRowGroup / 2;   // fp16 elements of a chunk's hi (or lo) part
  const int64_t total = int64_t(ig.nchunk) * 2 * per_half;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int64_t ch = e / (2 * per_half);
    const int64_t w = e % (2 * per_half);
    const int part = int(w / per_half);                  // 0 hi, 1 lo
    const int64_t x = w % per_half;
    const int grp = int(x / (kRowGroup / 2)), y = int(x % (kRowGroup / 2));
    const int kgi = y / 64, m = grp * 8 + (y / 8) % 8, k = kgi * 8 + y % 8;
    const int col = int(ch) * kKC + k / 2;
    float v = 0.f;
    if (m < ig.nrow && col < ig.nblk) {
      const float2 wv = src[int64_t(m) * ig.nblk + col];
      v = (k & 1 ? wv.y : wv.x) * srow[m];
    }
    __half hi, lo;
    split16(v, hi, lo);
    dst[e] = part == 0 ? hi : lo;
  }
}

}  // namespace

int64_t tc_tile_elems(int nrow, int nblk) {
  // hi and lo fp16 parts together take the bytes of the complex64 values
  const int groups = (std::min(nrow, kTcRows) + 7) / 8;
  return int64_t((nblk + kKC - 1) / kKC) * groups * (2 * kRowGroup / 8);
}

cudaError_t tile_weights(const ApplyData<float2>& d, float2* Wt, float* rscale, cudaStream_t st) {
  if (d.n_items128 == 0) return cudaSuccess;
  k_tile_weights<<<d.n_items128, 256, 0, st>>>(d.items128, d.tile_off, d.occ_start, d.blk_off, d.blk_seg, d.Wb,
                                               reinterpret_cast<unsigned char*>(Wt), rscale);
  return cudaGetLastError();
}

template <int R>
cudaError_t near_eval_tc(const ApplyData<float2>& d, const float2* u, float2* out, cudaStream_t st) {
  using Lay = TcLayout<R>;
  static unsigned long long attr = 0;
  static int n_sm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (first_on_device(attr)) {
    cudaError_t e = cudaFuncSetAttribute(k_near_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kBytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) {
      e = cudaDeviceGetAttribute(&n_sm[dev], cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
    }
  }
  if (d.n_items128 == 0) return cudaSuccess;
  cudaError_t e0 = cudaMemsetAsync(d.tc_tmax, 0, sizeof(unsigned) * R, st);
  if (e0 != cudaSuccess) return e0;
  k_rhs_max<<<dim3(kScaleBlocks, R), 256, 0, st>>>(u, d.N, d.tc_tmax);
  // the per-block item lists were balanced for the plan device's SM count
  const int sms = (dev >= 0 && dev < 64 && n_sm[dev] > 0) ? n_sm[dev] : 0;
  if (d.tc_grid <= 0 || d.tc_grid > sms || !d.tc_bptr || !d.tc_blist) return cudaErrorInvalidConfiguration;
  k_near_tc<R><<<d.tc_grid, kThreads, Lay::kBytes, st>>>(d.items128, d.tc_bptr, d.tc_blist, d.tile_off, d.occ_start, d.blk_seg,
                                                     reinterpret_cast<const unsigned char*>(d.Wt), d.tc_rscale,
                                                     d.tc_tmax, d.rem_row, d.rem_col, d.rem_val, u, d.N, d.Phi,
                                                     d.gamma, d.nocc, d.nfb2, float(d.kappa2), out, d.tc_err,
                                                     d.tc_spin);
  return cudaGetLastError();
}

template cudaError_t near_eval_tc<8>(const ApplyData<float2>&, const float2*, float2*, cudaStream_t);
template cudaError_t near_eval_tc<16>(const ApplyData<float2>&, const float2*, float2*, cudaStream_t);

}  // namespace lsd
