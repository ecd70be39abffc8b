// Local-expansion coefficients of R complex64 right-hand sides (R = 8 or 16)
// on the 5th-generation tensor cores (tcgen05, sm_103a): Section 3.2's
//   gamma_c = B^+ V_c - sum_o (B^+ T_o) sigma_{c+o}
// written, as on the CUDA cores, as one contraction per cell and right-hand
// side, gamma = LA X with LA = [B^+, -B^+ T_0, ..., -B^+ T_8] shared by every
// cell (nfb2 x K complex, K = (N_eq + 1)^2 + 9 n_es) and X = [V at the cell's
// lattice points; the 3 x 3 neighbours' strengths].
//
// One block takes 128 / R cells, so that the rows m = (cell, RHS) of
// X^T fill one MMA of M = 128:  D (128 x 64) = X^T (128 x 2K) . LA' (2K x 64),
// with X interleaved along K (A[m][2j] = Re x_j, A[m][2j + 1] = Im x_j) and
// the 64 columns of LA' holding, for output o < 32, (Re LA, -Im LA) in column o
// and (Im LA, Re LA) in column 32 + o, so that column o of D is Re gamma_o and
// column 32 + o is Im gamma_o.  3xTF32 (kind::tf32): every operand is split as
// x = hi + lo with hi = x with its 13 low mantissa bits cleared and lo = x - hi
// (exact in FP32; the tensor core reads the TF32 part of each word), and per
// K step of 8 one MMA A_hi . [B_hi | B_lo] (N = 128) and one A_lo . B_hi
// (N = 64) accumulate into the same FP32 accumulator; the epilogue adds
// column n and column 64 + n.  TF32 keeps FP32's exponent, so no scaling is
// needed (the split-FP16 near field needs power-of-two scales).
//
// A block: all 256 threads build the A chunk (16 complex columns, hi and lo)
// from the lattice values and strengths and copy the LA' chunk (stored in the
// tile layout at plan time) into one of two shared-memory stages; thread 0
// issues the chunk's MMAs and commits them to the stage's mbarrier, which
// the block waits on (bounded) before it refills the stage two chunks later.
// Warps 0..3 read the accumulator (lane = row) and write gamma.
#include <cstdint>

#include <cuda_fp16.h>

#include "device/cplx.cuh"
#include "device/kernels.cuh"

namespace lsd {
namespace {

constexpr int kLT = 256;                 // threads
constexpr int kLChunk = 16;              // complex K columns per chunk (32 real: four K steps of 8)
constexpr int kLGroup = 1024;            // bytes of one 8-row group of a chunk (8 core-matrix columns x 128)
constexpr int kLA = 16 * kLGroup;        // 128 rows of A, hi or lo: 16 KB
constexpr int kLB = 16 * kLGroup;        // LA' chunk: 64 hi rows then 64 lo rows: 16 KB
constexpr int kLStage = 2 * kLA + kLB;   // one pipeline stage: A hi, A lo, LA'
constexpr int kLSmem = 2 * kLStage + 64;
constexpr int kLDrain = 1 << 28;         // bound of the final wait on the block's own MMAs

__device__ __forceinline__ uint32_t ls_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// K-major, no swizzle: 128 bytes between K-adjacent core matrices, kLGroup between row groups
__device__ __forceinline__ uint64_t ls_desc(uint32_t addr) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((128 >> 4) & 0x3FFF) << 16) |
         (uint64_t((kLGroup >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

__device__ __forceinline__ bool lbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// 16 consecutive accumulator columns of this thread's lane (load and wait in one statement)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* d) {
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

// byte offset of FP32 element (row n, real column k) of a chunk in the
// K-major core-matrix layout (8 rows x 16 bytes = 4 elements per core matrix)
__device__ __forceinline__ int lt_off(int n, int k) {
  return (n >> 3) * kLGroup + (k >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

// x = hi + lo: hi keeps the 10 mantissa bits TF32 reads, lo = x - hi (exact)
__device__ __forceinline__ void tsplit(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

template <int R>
__global__ void __launch_bounds__(kLT) k_local_tc(ApplyData<float2> d, const float2* __restrict__ V, int64_t stride,
                                                  const unsigned char* __restrict__ LAt, int spin) {
  constexpr int G = 128 / R;                    // cells per block
  extern __shared__ __align__(1024) unsigned char lsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(lsm + 2 * kLStage);   // MMAs of the stage's chunk done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  int* flag = reinterpret_cast<int*>(tslot + 1);
  __shared__ int cij[G][2];                     // the block's cells: lattice coordinates
  __shared__ int nb9[G][9];                     // occupied index of each neighbour (o = 3 di + dj), or -1
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int K = d.n_loc + 9 * d.n_es, nch = (K + kLChunk - 1) / kLChunk;
  const int k0 = blockIdx.x * G, n1 = d.Ne + 1;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(ls_u32(tslot)), "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(ls_u32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(ls_u32(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *flag = 0;
  }
  if (t < G * 9) {
    const int g = t / 9, o = t % 9, k = k0 + g;
    int occ = -1;
    if (k < d.nocc) {
      const int c = d.occ_cells[k], ci = c % d.L, cj = c / d.L;
      if (o == 0) { cij[g][0] = ci; cij[g][1] = cj; }
      const int ni = ci + o / 3 - 1, nj = cj + o % 3 - 1;
      if (ni >= 0 && ni < d.L && nj >= 0 && nj < d.L) occ = d.occ_of_cell[nj * d.L + ni];
    }
    nb9[g][o] = occ;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // kind::tf32: D F32, A and B TF32, both K-major; M = 128, N = 128 or 64
  const uint32_t idesc1 = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(128 >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  const uint32_t idesc2 = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(64 >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  int issued = -1;                              // last chunk whose MMAs thread 0 committed

  // the inputs of chunk c (X values and LA' words) are loaded into registers
  // during chunk c - 1, so that their latency overlaps the barriers and the
  // wait for the MMAs of chunk c - 2
  constexpr int kXv = (128 * kLChunk) / kLT, kBv = kLB / 16 / kLT;
  float2 xv[kXv];
  uint4 bv[kBv];
  auto load_chunk = [&](int c) {
#pragma unroll
    for (int i = 0; i < kXv; ++i) {
      const int v = t + i * kLT, m = v >> 4, jj = v & 15, g = m / R, r = m % R, j = c * kLChunk + jj;
      float2 x = make_float2(0.f, 0.f);
      if (k0 + g < d.nocc && j < K) {
        if (j < d.n_loc) {
          const int a = j / n1, b = j - a * n1;
          x = V[int64_t(r) * stride + int64_t(cij[g][0] * d.Ne + a) * d.M + cij[g][1] * d.Ne + b];
        } else {
          const int q = j - d.n_loc, o = q / d.n_es, l = q - o * d.n_es, occ = nb9[g][o];
          if (occ >= 0) x = d.sigma[(int64_t(r) * d.nocc + occ) * d.n_es + l];
        }
      }
      xv[i] = x;
    }
    const uint4* src = reinterpret_cast<const uint4*>(LAt + int64_t(c) * kLB);
#pragma unroll
    for (int i = 0; i < kBv; ++i) bv[i] = src[t + i * kLT];
  };
  load_chunk(0);
  for (int c = 0; c < nch; ++c) {
    const int s = c & 1;
    if (c >= 2 && t == 0) {                     // the MMAs of chunk c - 2 have read stage s
      bool ok = false;
      for (int it = 0; it < spin && !ok; ++it) ok = lbar_try(ls_u32(&bar[s]), uint32_t((c - 2) >> 1) & 1u);
      if (!ok) *flag = 1;
    }
    __syncthreads();
    if (*flag) break;
    unsigned char* Ahi = lsm + s * kLStage;
    unsigned char* Alo = Ahi + kLA;
    unsigned char* Bs = Ahi + 2 * kLA;
#pragma unroll
    for (int i = 0; i < kBv; ++i) reinterpret_cast<uint4*>(Bs)[t + i * kLT] = bv[i];
#pragma unroll
    for (int i = 0; i < kXv; ++i) {
      const int v = t + i * kLT, m = v >> 4, jj = v & 15;
      float rh, rl, ih, il;
      tsplit(xv[i].x, rh, rl);
      tsplit(xv[i].y, ih, il);
      *reinterpret_cast<float2*>(Ahi + lt_off(m, 2 * jj)) = make_float2(rh, ih);
      *reinterpret_cast<float2*>(Alo + lt_off(m, 2 * jj)) = make_float2(rl, il);
    }
    if (c + 1 < nch) load_chunk(c + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = ls_u32(Ahi), b0 = ls_u32(Bs);
#pragma unroll
      for (int i = 0; i < 4; ++i) {             // K = 8 per MMA: core-matrix columns 2i, 2i + 1
        const uint64_t dh = ls_desc(a0 + 2 * i * 128), dl = ls_desc(a0 + kLA + 2 * i * 128);
        const uint64_t db = ls_desc(b0 + 2 * i * 128);
        const uint32_t accum = (c > 0 || i > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tmem), "l"(dh), "l"(db), "r"(idesc1), "r"(accum) : "memory");
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tmem), "l"(dl), "l"(db), "r"(idesc2), "r"(1u) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(ls_u32(&bar[s])) : "memory");
      issued = c;
    }
  }
  // the last commit tracks every MMA of the block: wait for it (fixed bound)
  // before the accumulator is read or freed
  if (t == 0 && issued >= 0) {
    bool ok = false;
    for (int it = 0; it < kLDrain && !ok; ++it) ok = lbar_try(ls_u32(&bar[issued & 1]), uint32_t(issued >> 1) & 1u);
    if (!ok || issued != nch - 1) *flag = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool good = *flag == 0;
  if (!good && t == 0) atomicExch(d.tc_err, 1);
  if (good && warp < 4) {
    const int m = 32 * warp + lane, g = m / R, r = m % R, k = k0 + g;
    const uint32_t ta = tmem + (uint32_t(32 * warp) << 16);
#pragma unroll
    for (int ob = 0; ob < 32; ob += 16) {
      float re_h[16], re_l[16], im_h[16], im_l[16];
      tmem_ld16(ta + uint32_t(ob), re_h);
      tmem_ld16(ta + uint32_t(64 + ob), re_l);
      tmem_ld16(ta + uint32_t(32 + ob), im_h);
      tmem_ld16(ta + uint32_t(96 + ob), im_l);
      if (k < d.nocc) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int o = ob + i;
          if (o < d.nfb2)
            d.gamma[(int64_t(r) * d.nocc + k) * d.nfb2 + o] = make_float2(re_h[i] + re_l[i], im_h[i] + im_l[i]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(128) : "memory");
  }
}

// Equivalent-source projection (Section 3.2: the strengths of cell c solve the
// fit to the scaled field on the cell's nodes, sigma_c = P_c u_c with P_c the
// fit's pseudo-inverse folded with the quadrature weights) for R = 8 or 16
// right-hand sides:  one block per occupied cell (largest first),
// D (128 x 2R) = P' (128 x 2n) . [u_hi | u_lo] (2n x 2R) with u
// interleaved along K (B[r][2j] = Re u_j, B[r][2j + 1] = Im u_j, the layout of
// u in memory) and the rows of P' built from P_c as it is stored ([node][n_es]):
// row i < n_es holds (Re P, -Im P) of output i, row 64 + i holds (Im P, Re P),
// so row i of D is Re sigma_i and row 64 + i is Im sigma_i.  Rows n_es..63
// and 64 + n_es..127 are zero.  3xTF32 as in the local step, here with both
// MMAs on [B_hi | B_lo] (N = 2R: an MMA of M = 128 needs N >= 16, so the
// A_lo . B_lo product of R = 8 comes for free; the epilogue adds columns r and
// R + r).  Nodes are taken 16 per chunk (K = 32 real, four K steps of 8).
// Whole cells, unlike the CUDA-core projection's pieces of at most 128 nodes:
// the tensor cores take a long cell in stride, and without partial sums no
// block waits on a merge (pieces with a merge ran 8% slower).
constexpr int kPB = 4096;                // B chunk: 2R <= 32 rows x 128 bytes
constexpr int kPStage = 2 * kLA + kPB;   // one pipeline stage: P' hi, P' lo, [u_hi | u_lo]
constexpr int kPSmem = 2 * kPStage + 64;

template <int R>
__global__ void __launch_bounds__(kLT) k_project_tc(const int4* __restrict__ cells, int nocc,
                                                    const int64_t* __restrict__ occ_start,
                                                    const int64_t* __restrict__ P_off, const float2* __restrict__ P,
                                                    const float2* __restrict__ u, int64_t N,
                                                    float2* __restrict__ sigma, int n_es, int* __restrict__ tc_err,
                                                    int spin) {
  extern __shared__ __align__(1024) unsigned char psm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(psm + 2 * kPStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  int* flag = reinterpret_cast<int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int k = cells[blockIdx.x].x;            // (cell, 0, nodes, 1)
  const int64_t s0 = occ_start[k];
  const int nc = int(occ_start[k + 1] - s0), nch = (nc + kLChunk - 1) / kLChunk;
  const float2* Pk = P + P_off[k];

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(ls_u32(tslot)), "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(ls_u32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(ls_u32(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *flag = 0;
  }
  // zero the rows of P' that no output uses, in both stages (hi and lo)
  for (int e = t; e < 2 * 2 * 2 * (64 - n_es) * 16; e += kLT) {
    const int w = e & 15, row = (e >> 4) % (64 - n_es), q = (e >> 4) / (64 - n_es);   // q: stage, half, hi / lo
    unsigned char* A = psm + (q >> 2) * kPStage + (q & 1) * kLA;
    const int n = n_es + row + ((q >> 1) & 1) * 64;
    *reinterpret_cast<float2*>(A + lt_off(n, 2 * w)) = make_float2(0.f, 0.f);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // kind::tf32: D F32, A and B TF32, both K-major; M = 128, N = 2R
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t((2 * R) >> 3) << 17) |
                         (uint32_t(128 >> 4) << 24);
  int issued = -1;

  // the inputs of two chunks are in flight in registers: chunk c + 2 is loaded
  // into the set chunk c was just stored from.  A warp takes 16 outputs x 2
  // nodes of P (and 8 RHS x 4 nodes of u), so that its 8-byte shared-memory
  // stores fall on every bank twice
  constexpr int kPv = 4;                        // 8 node pairs x 4 blocks of 16 outputs x 32 / 256
  const int nob = (n_es + 15) >> 4;
  float2 pa[kPv], pb[kPv], ua = make_float2(0.f, 0.f), ub = make_float2(0.f, 0.f);
  auto p_slot = [&](int i, int& o, int& jj) {
    const int sl = t + i * kLT, unit = sl >> 5, ln = sl & 31;
    o = (unit % nob) * 16 + (ln & 15);
    jj = 2 * (unit / nob) + (ln >> 4);
    return unit < 8 * nob && o < n_es;
  };
  const int ur = (lane & 7) + 8 * (warp % (R / 8)), ujj = (lane >> 3) + 4 * (warp / (R / 8));
  auto load_chunk = [&](int c, float2 (&pv)[kPv], float2& uv) {
#pragma unroll
    for (int i = 0; i < kPv; ++i) {
      int o, jj;
      const bool ok = p_slot(i, o, jj) && c * kLChunk + jj < nc;
      pv[i] = ok ? Pk[int64_t(c * kLChunk + jj) * n_es + o] : make_float2(0.f, 0.f);
    }
    const int j = c * kLChunk + ujj;
    uv = (t < R * kLChunk && j < nc) ? u[int64_t(ur) * N + s0 + j] : make_float2(0.f, 0.f);
  };
  // wait until stage c & 1 is free, then split chunk c into it; false: a wait gave up
  auto store_chunk = [&](int c, const float2 (&pv)[kPv], const float2& uv) {
    const int s = c & 1;
    if (c >= 2 && t == 0) {                     // the MMAs of chunk c - 2 have read stage s
      bool ok = false;
      for (int it = 0; it < spin && !ok; ++it) ok = lbar_try(ls_u32(&bar[s]), uint32_t((c - 2) >> 1) & 1u);
      if (!ok) *flag = 1;
    }
    __syncthreads();
    if (*flag) return false;
    unsigned char* Ahi = psm + s * kPStage;
    unsigned char* Alo = Ahi + kLA;
    unsigned char* Bs = Ahi + 2 * kLA;
#pragma unroll
    for (int i = 0; i < kPv; ++i) {
      int o, jj;
      if (p_slot(i, o, jj)) {
        float rh, rl, ih, il;
        tsplit(pv[i].x, rh, rl);
        tsplit(pv[i].y, ih, il);
        *reinterpret_cast<float2*>(Ahi + lt_off(o, 2 * jj)) = make_float2(rh, -ih);
        *reinterpret_cast<float2*>(Ahi + lt_off(64 + o, 2 * jj)) = make_float2(ih, rh);
        *reinterpret_cast<float2*>(Alo + lt_off(o, 2 * jj)) = make_float2(rl, -il);
        *reinterpret_cast<float2*>(Alo + lt_off(64 + o, 2 * jj)) = make_float2(il, rl);
      }
    }
    if (t < R * kLChunk) {
      float rh, rl, ih, il;
      tsplit(uv.x, rh, rl);
      tsplit(uv.y, ih, il);
      *reinterpret_cast<float2*>(Bs + lt_off(ur, 2 * ujj)) = make_float2(rh, ih);
      *reinterpret_cast<float2*>(Bs + lt_off(R + ur, 2 * ujj)) = make_float2(rl, il);
    }
    return true;
  };
  // thread 0 issues chunk c's MMAs once every thread has stored it
  auto issue_chunk = [&](int c) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      const int s = c & 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = ls_u32(psm + s * kPStage), b0 = a0 + 2 * kLA;
#pragma unroll
      for (int i = 0; i < 4; ++i) {             // K = 8 per MMA: core-matrix columns 2i, 2i + 1
        const uint64_t dh = ls_desc(a0 + 2 * i * 128), dl = ls_desc(a0 + kLA + 2 * i * 128);
        const uint64_t db = ls_desc(b0 + 2 * i * 128);
        const uint32_t accum = (c > 0 || i > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tmem), "l"(dh), "l"(db), "r"(idesc), "r"(accum) : "memory");
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tmem), "l"(dl), "l"(db), "r"(idesc), "r"(1u) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(ls_u32(&bar[s])) : "memory");
      issued = c;
    }
  };
  if (nch > 0) load_chunk(0, pa, ua);
  if (nch > 1) load_chunk(1, pb, ub);
  for (int c = 0; c < nch; c += 2) {
    if (!store_chunk(c, pa, ua)) break;
    if (c + 2 < nch) load_chunk(c + 2, pa, ua);
    issue_chunk(c);
    if (c + 1 >= nch) break;
    if (!store_chunk(c + 1, pb, ub)) break;
    if (c + 3 < nch) load_chunk(c + 3, pb, ub);
    issue_chunk(c + 1);
  }
  if (t == 0 && issued >= 0) {
    bool ok = false;
    for (int it = 0; it < kLDrain && !ok; ++it) ok = lbar_try(ls_u32(&bar[issued & 1]), uint32_t(issued >> 1) & 1u);
    if (!ok || issued != nch - 1) *flag = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool good = *flag == 0 && nch > 0;
  if (*flag && t == 0 && tc_err) atomicExch(tc_err, 1);
  float2* out = sigma + int64_t(k) * n_es;      // sigma: [r][cell][i]
  const int64_t rs = int64_t(nocc) * n_es;
  if (warp < 4) {
    const int m = 32 * warp + lane, o = m & 63, im = m >> 6;
    float v[2 * R];
    if (good) {
      const uint32_t ta = tmem + (uint32_t(32 * warp) << 16);
#pragma unroll
      for (int q = 0; q < 2 * R; q += 16) tmem_ld16(ta + uint32_t(q), v + q);
    } else {
#pragma unroll
      for (int q = 0; q < 2 * R; ++q) v[q] = 0.f;
    }
    if (o < n_es) {
#pragma unroll
      for (int r = 0; r < R; ++r) reinterpret_cast<float*>(out + r * rs + o)[im] = v[r] + v[R + r];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(32) : "memory");
  }
}

// plan time: LA' in the tile layout, per chunk of 16 complex K columns the 64
// hi rows then the 64 lo rows (row n < 32: (Re, -Im) of output n; 32 <= n < 64:
// (Im, Re) of output n - 32), zero past K or nfb2
__global__ void __launch_bounds__(kLT) k_la_tiles(const float2* __restrict__ LA, int K, int nfb2,
                                                  unsigned char* __restrict__ LAt, int nch) {
  const int64_t total = int64_t(nch) * 128 * 32;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(e / (128 * 32)), n = int((e / 32) % 128), k = int(e % 32);
    const int part = n >> 6, nn = n & 63, o = nn & 31, imcol = nn >> 5;
    const int j = c * kLChunk + k / 2, comp = k & 1;
    float v = 0.f;
    if (o < nfb2 && j < K) {
      const float2 l = LA[int64_t(j) * nfb2 + o];
      v = imcol == 0 ? (comp == 0 ? l.x : -l.y) : (comp == 0 ? l.y : l.x);
    }
    float hi, lo;
    tsplit(v, hi, lo);
    *reinterpret_cast<float*>(LAt + int64_t(c) * kLB + lt_off(n, k)) = part == 0 ? hi : lo;   // lo: rows 64..127
  }
}

}  // namespace

int local_tc_chunks(int K) { return (K + kLChunk - 1) / kLChunk; }

size_t local_tc_bytes(int K) { return size_t(local_tc_chunks(K)) * kLB; }

cudaError_t local_tc_tiles(const float2* LA, int K, int nfb2, unsigned char* LAt, cudaStream_t st) {
  if (nfb2 > 32 || K <= 0) return cudaErrorInvalidValue;
  const int nch = local_tc_chunks(K);
  k_la_tiles<<<(nch * 128 * 32 + kLT - 1) / kLT, kLT, 0, st>>>(LA, K, nfb2, LAt, nch);
  return cudaGetLastError();
}

template <int R>
cudaError_t local_coeffs_tc(const ApplyData<float2>& d, cudaStream_t st) {
  static unsigned long long attr = 0;
  if (first_on_device(attr)) {
    const cudaError_t e = cudaFuncSetAttribute(k_local_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLSmem);
    if (e != cudaSuccess) return e;
  }
  if (!d.LAt || d.nfb2 > 32 || d.nocc <= 0) return cudaErrorInvalidValue;
  constexpr int G = 128 / R;
  k_local_tc<R><<<(d.nocc + G - 1) / G, kLT, kLSmem, st>>>(d, d.Sd, d.lattice_rows() * d.M, d.LAt, d.tc_spin);
  return cudaGetLastError();
}

template cudaError_t local_coeffs_tc<8>(const ApplyData<float2>&, cudaStream_t);
template cudaError_t local_coeffs_tc<16>(const ApplyData<float2>&, cudaStream_t);

template <int R>
cudaError_t project_tc(const ApplyData<float2>& d, const float2* u, cudaStream_t st) {
  static unsigned long long attr = 0;
  if (first_on_device(attr)) {
    const cudaError_t e = cudaFuncSetAttribute(k_project_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem);
    if (e != cudaSuccess) return e;
  }
  if (d.n_es <= 0 || d.n_es > 64 || d.nocc <= 0 || !d.cell_pieces) return cudaErrorInvalidValue;
  // one block per whole cell, largest first (d.cell_pieces)
  k_project_tc<R><<<d.nocc, kLT, kPSmem, st>>>(d.cell_pieces, d.nocc, d.occ_start, d.P_off, d.P, u, d.N, d.sigma,
                                               d.n_es, d.tc_err, d.tc_spin);
  return cudaGetLastError();
}

template cudaError_t project_tc<8>(const ApplyData<float2>&, const float2*, cudaStream_t);
template cudaError_t project_tc<16>(const ApplyData<float2>&, const float2*, cudaStream_t);

}  // namespace lsd
