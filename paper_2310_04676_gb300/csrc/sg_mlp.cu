// Dense contraction of the PPO networks on the 5th-generation tensor cores
// (tcgen05), FP32-grade by splitting every operand into two TF32 parts.
//
//   C[m][n] = epi( sum_k A(m, k) B(n, k) ),  A(m, k) = A[m a_m + k a_k],
//                                            B(n, k) = B[n b_n + k b_k]
//
// With general strides the one kernel serves the three products of a layer
// (rows = minibatch rows, W = [out][in]):
//   forward        Y  = ELU(X W^T + b)  A = X  (k = in),   B = W  (n = out, k = in)
//   input grad     dZ = (dY W) ELU'(y)  A = dY (k = out),  B = W^T (n = in, k = out),
//                                       with the column sums of dZ (the bias
//                                       gradient of the layer below) per row tile
//   weight grad    dW = dY^T X          A = dY^T (m = out, k = row), B = X^T (n = in, k = row),
//                                       the rows split over CTAs (partial sums,
//                                       then a fixed-order reduction: results do
//                                       not depend on scheduling).
//
// Split precision (3xTF32): x = hi + lo with hi = tf32(x) and lo = tf32(x - hi);
// a b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b, the dropped lo_a lo_b term being
// about 2^-22 of a b, so the products carry FP32 accuracy with FP32
// accumulation (the published "3xTF32" emulation of FP32 matrix products).
//
// One CTA of 128 threads computes a 128 x Nt tile (Nt <= 128, a multiple of
// 16).  Raw FP32 operand chunks (16 wide in K) travel to shared memory by
// asynchronous copies three chunks ahead; each chunk is then split into its
// TF32 parts and stored in the tensor cores' K-major layout without swizzle
// (8-row x 16-byte core matrices).  One thread issues, per 8-wide K step, the
// three tcgen05.mma of kind::tf32 into an FP32 accumulator in tensor memory
// (TMEM lane = row, column = n) and commits them to an mbarrier; two
// tensor-core stages alternate, a stage being refilled only after the
// mbarrier of the MMAs that read it has completed (bounded wait).  The
// epilogue reads the accumulator with tcgen05.ld (each warp its 32 TMEM
// lanes), applies the epilogue and stores whole row segments.
#include <cuda_runtime.h>

#include <cstdint>

#include "sg.h"
#include "sg_internal.h"
#include "sg_mlp.h"

namespace sg {
namespace {

constexpr int kMlpThreads = 128;
constexpr int kTileM = 128;
constexpr int kChunkK = 16;                       // K per shared-memory chunk (2 MMA K-steps)
constexpr int kCoreBytes = 128;                   // one core matrix: 8 rows x 16 bytes
constexpr int kLbo = kCoreBytes;                  // next core matrix along K
constexpr int kSbo = (kChunkK / 4) * kCoreBytes;  // next 8-row group (512 bytes)
constexpr unsigned long long kMmaWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of a tile (rows r, K within the chunk) in
// the K-major no-swizzle layout.
__device__ __forceinline__ unsigned tile_off(int r, int k) {
  return (unsigned)((r >> 3) * kSbo + (k >> 2) * kLbo + (r & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// and stride (8-row group) byte offsets in 16-byte units, descriptor
// version 1 (bits 46-47), no swizzle (layout type 0, bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(unsigned addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kLbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kSbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_poll(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for phase `parity` (wall-clock limit, iteration cap).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_poll(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 0; it < (1u << 24); ++it) {
    if (mbar_poll(bar, parity)) return true;
    if (gtimer() - t0 > kMmaWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate ? 1 : 0)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- operand chunks ---------------------------------------------------------
// Rows [r0, r0 + nrows) x K [k0, k0 + 16) of X(r, k) = X[r xr + k xk] (zero
// outside R x K).  Raw chunks travel to shared memory by asynchronous
// 16-byte copies (cp.async, zero-filled outside the operand), kRawStages - 1
// chunks ahead, in whichever layout is contiguous in global memory:
// row-major [r][16] when K is the contiguous direction (xk = 1), K-major
// [16][nrows] when the rows are (xr = 1); other strides are read by plain
// loads.  The conversion then cuts the chunk into 4-element units (row r, K
// group kg) numbered core matrix by core matrix -- unit f has
// r = 8 (f >> 5) + (f & 7), kg = (f >> 3) & 3, so eight consecutive threads
// store the eight rows of one core matrix (conflict-free 16-byte stores) --
// splits each value into its TF32 parts and stores them to the tiles.
constexpr int kRawStages = 3;
constexpr int kMaxTileN = 128;
constexpr int kUnitsA = kTileM * (kChunkK / 4) / kMlpThreads;      // 4 per thread
constexpr int kUnitsB = kMaxTileN * (kChunkK / 4) / kMlpThreads;   // at most 4 per thread

enum RawLayout { RAW_ROWS = 0, RAW_KMAJOR = 1, RAW_PLAIN = 2 };

struct Operand {
  const float* X;
  long long xr, xk;
  int R, K, r0, nrows, layout;
};

__device__ __forceinline__ Operand make_operand(const float* X, long long xr, long long xk, int R,
                                                int K, int r0, int nrows) {
  Operand o{X, xr, xk, R, K, r0, nrows, RAW_PLAIN};
  const bool al = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (al && xk == 1 && (xr & 3) == 0) o.layout = RAW_ROWS;
  else if (al && xr == 1 && (xk & 3) == 0 && (nrows & 3) == 0) o.layout = RAW_KMAJOR;
  return o;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the asynchronous copies of chunk k0 of an operand into raw.
__device__ __forceinline__ void raw_issue(const Operand& o, int k0, float* raw, int tid) {
  if (o.layout == RAW_ROWS) {
    for (int u = tid; u < o.nrows * 4; u += kMlpThreads) {
      const int r = u >> 2, kg = u & 3;
      const int gr = o.r0 + r, gk = k0 + 4 * kg;
      const int nk = gr < o.R ? max(0, min(4, o.K - gk)) : 0;
      const float* src = nk ? o.X + (long long)gr * o.xr + gk : o.X;
      cp_async16(raw + r * kChunkK + 4 * kg, src, 4 * nk);
    }
  } else if (o.layout == RAW_KMAJOR) {
    const int rg = o.nrows >> 2;
    for (int u = tid; u < kChunkK * rg; u += kMlpThreads) {
      const int k = u / rg, q = u - k * rg;
      const int gk = k0 + k, gr = o.r0 + 4 * q;
      const int nr = gk < o.K ? max(0, min(4, o.R - gr)) : 0;
      const float* src = nr ? o.X + (long long)gk * o.xk + gr : o.X;
      cp_async16(raw + k * o.nrows + 4 * q, src, 4 * nr);
    }
  }
}

// Convert chunk k0 (from raw, or read directly for RAW_PLAIN) into the
// hi / lo tiles.
template <int U>
__device__ __forceinline__ void convert(const Operand& o, int k0, const float* raw, int tid,
                                        char* hi, char* lo) {
  const int units = o.nrows * (kChunkK / 4);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int f = tid + u * kMlpThreads;
    if (f >= units) continue;
    const int r = ((f >> 5) << 3) + (f & 7), kg = (f >> 3) & 3;
    float v[4];
    if (o.layout == RAW_ROWS) {
      const float4 t = *reinterpret_cast<const float4*>(raw + r * kChunkK + 4 * kg);
      v[0] = t.x;
      v[1] = t.y;
      v[2] = t.z;
      v[3] = t.w;
    } else if (o.layout == RAW_KMAJOR) {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = raw[(4 * kg + j) * o.nrows + r];
    } else {
      const int gr = o.r0 + r;
      const float* row = o.X + (long long)gr * o.xr;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gk = k0 + 4 * kg + j;
        v[j] = (gr < o.R && gk < o.K) ? __ldg(row + (long long)gk * o.xk) : 0.f;
      }
    }
    float4 h, l;
    h.x = to_tf32(v[0]);
    h.y = to_tf32(v[1]);
    h.z = to_tf32(v[2]);
    h.w = to_tf32(v[3]);
    l.x = to_tf32(v[0] - h.x);
    l.y = to_tf32(v[1] - h.y);
    l.z = to_tf32(v[2] - h.z);
    l.w = to_tf32(v[3] - h.w);
    const unsigned off = tile_off(r, kg * 4);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}

// Epilogue modes (compile-time, no per-element branches): plain product,
// bias (+ ELU), ELU only, or the ELU derivative of the layer below with
// column sums.
enum EpiMode { EPI_PLAIN = 0, EPI_BIAS = 1, EPI_BIAS_ELU = 2, EPI_DELU_SUM = 3, EPI_ELU = 4 };

// ELU from the hardware exponential: e^x - 1 for x <= 0 (absolute error
// about 1e-7 against expm1; the layers' activations are O(1))
__device__ __forceinline__ float elu_fast(float x) { return x > 0.f ? x : __expf(x) - 1.f; }

template <int kEpi>
__global__ void __launch_bounds__(kMlpThreads) mlp_gemm_kernel(MlpGemmArgs g) {
  extern __shared__ __align__(1024) char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Nt = g.n_tile;                         // multiple of 16, <= 128
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * Nt;
  const int kbeg = blockIdx.z * g.k_per_split;
  const int kend = min(g.K, kbeg + g.k_per_split);
  const int a_bytes = kTileM * kChunkK * 4, b_bytes = Nt * kChunkK * 4;
  const int stage_bytes = 2 * (a_bytes + b_bytes);
  // two tensor-core stages of (A hi, A lo, B hi, B lo), then kRawStages raw
  // stages of (A, B)
  auto a_hi = [&](int st) { return sm + st * stage_bytes; };
  auto a_lo = [&](int st) { return sm + st * stage_bytes + a_bytes; };
  auto b_hi = [&](int st) { return sm + st * stage_bytes + 2 * a_bytes; };
  auto b_lo = [&](int st) { return sm + st * stage_bytes + 2 * a_bytes + b_bytes; };
  char* raw0 = sm + 2 * stage_bytes;
  auto raw_a = [&](int st) { return reinterpret_cast<float*>(raw0 + st * (a_bytes + b_bytes)); };
  auto raw_b = [&](int st) {
    return reinterpret_cast<float*>(raw0 + st * (a_bytes + b_bytes) + a_bytes);
  };
  uint64_t* bar = reinterpret_cast<uint64_t*>(raw0 + kRawStages * (a_bytes + b_bytes));   // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t ncols = Nt <= 32 ? 32u : (Nt <= 64 ? 64u : 128u);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init1(bar);
    mbar_init1(bar + 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(kTileM, Nt);

  bool ok = true;
  // commits issued and completions awaited per stage barrier; a barrier is
  // awaited before its next commit, so it never holds two unawaited
  // completions and a parity wait is unambiguous
  int issued[2] = {0, 0}, waited[2] = {0, 0};
  const int nchunks = kbeg < kend ? (kend - kbeg + kChunkK - 1) / kChunkK : 0;
  const Operand opa = make_operand(g.A, g.a_m, g.a_k, g.M, g.K, m0, kTileM);
  const Operand opb = make_operand(g.B, g.b_n, g.b_k, g.N, g.K, n0, Nt);
  // prologue: the first kRawStages - 1 chunks in flight
#pragma unroll
  for (int c = 0; c < kRawStages - 1; ++c) {
    if (c < nchunks) {
      raw_issue(opa, kbeg + c * kChunkK, raw_a(c), tid);
      raw_issue(opb, kbeg + c * kChunkK, raw_b(c), tid);
    }
    cp_async_commit();
  }
  for (int c = 0; c < nchunks; ++c) {
    const int st = c & 1, rs = c % kRawStages;
    cp_async_wait<kRawStages - 2>();              // this thread's copies of chunk c landed
    __syncthreads();                              // ... and every thread's
    {
      const int cn = c + kRawStages - 1;          // refill the stage chunk c - 1 came from
      if (cn < nchunks) {
        raw_issue(opa, kbeg + cn * kChunkK, raw_a(cn % kRawStages), tid);
        raw_issue(opb, kbeg + cn * kChunkK, raw_b(cn % kRawStages), tid);
      }
      cp_async_commit();
    }
    // tensor-core stage st was read by the MMAs of chunk c - 2
    if (waited[st] < issued[st]) {
      const bool done = __syncthreads_and(mbar_wait(bar + st, (unsigned)waited[st] & 1u));
      if (!done) {
        ok = false;
        break;
      }
      ++waited[st];
    }
    convert<kUnitsA>(opa, kbeg + c * kChunkK, raw_a(rs), tid, a_hi(st), a_lo(st));
    convert<kUnitsB>(opb, kbeg + c * kChunkK, raw_b(rs), tid, b_hi(st), b_lo(st));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < kChunkK / 8; ++ks) {
        const unsigned koff = (unsigned)ks * 2 * kLbo;   // two core matrices per K step
        const uint64_t ah = smem_desc(smem_addr(a_hi(st)) + koff);
        const uint64_t al = smem_desc(smem_addr(a_lo(st)) + koff);
        const uint64_t bh = smem_desc(smem_addr(b_hi(st)) + koff);
        const uint64_t bl = smem_desc(smem_addr(b_lo(st)) + koff);
        mma_tf32(tmem, ah, bh, idesc, c > 0 || ks > 0);
        if (g.split_tf32) {
          mma_tf32(tmem, ah, bl, idesc, true);
          mma_tf32(tmem, al, bh, idesc, true);
        }
      }
      mma_commit(bar + st);
    }
    ++issued[st];
  }
  cp_async_wait<0>();
  // every MMA has completed once both barriers' last commits have
  for (int b = 0; b < 2 && ok; ++b) {
    if (waited[b] < issued[b]) {
      ok = __syncthreads_and(mbar_wait(bar + b, (unsigned)waited[b] & 1u));
      if (ok) ++waited[b];
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok && nchunks > 0) {
    // epilogue: warp w holds rows m0 + 32 w + lane (TMEM lanes 32 w ..).
    // Per 16 columns each thread finishes its row's values (bias, ELU, or the
    // ELU derivative of the layer below) and parks them in a shared-memory
    // slab of the warp (row pitch 20 floats).  From the slab the warp sums
    // the columns (lane l: column l % 16 over 16 rows, then the two halves;
    // fixed order) into its per-warp partials, and stores whole 64-byte row
    // segments, four lanes per row, eight rows per instruction (scalar stores
    // at ragged edges or unaligned outputs).  After the last slab the four
    // warps' partials are added in order.
    const int m = m0 + warp * 32 + lane;
    const bool mrow = m < g.M;
    float* cbase = g.C + (long long)blockIdx.z * g.c_split;
    float* slab = reinterpret_cast<float*>(sm) + warp * 32 * 20;
    float* wsum = reinterpret_cast<float*>(sm) + 4 * 32 * 20;          // [4][128]
    const bool cvec = (g.c_m & 3) == 0 && (reinterpret_cast<uintptr_t>(cbase) & 15) == 0;
    const bool yvec = kEpi == EPI_DELU_SUM && (g.c_m & 3) == 0 &&
                      (reinterpret_cast<uintptr_t>(g.act_y) & 15) == 0;
    for (int c = 0; c < Nt; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      const int ncol = min(16, g.N - (n0 + c));
      if (kEpi == EPI_DELU_SUM) {
        float y[16];
        const float* yr = g.act_y + (long long)m * g.c_m + n0 + c;
        if (yvec && mrow && ncol == 16) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(yr) + q);
            y[4 * q] = t.x;
            y[4 * q + 1] = t.y;
            y[4 * q + 2] = t.z;
            y[4 * q + 3] = t.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) y[j] = (mrow && j < ncol) ? yr[j] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] *= y[j] > 0.f ? 1.f : y[j] + 1.f;
      }
      if (kEpi == EPI_BIAS || kEpi == EPI_BIAS_ELU) {
        if (ncol == 16) {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += __ldg(g.bias + n0 + c + j);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += j < ncol ? __ldg(g.bias + n0 + c + j) : 0.f;
        }
      }
      if (kEpi == EPI_BIAS_ELU || kEpi == EPI_ELU) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = elu_fast(v[j]);
      }
      if (kEpi == EPI_DELU_SUM) {
        // rows and columns outside C add nothing to the column sums
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = (mrow && j < ncol) ? v[j] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(slab + lane * 20 + 4 * q) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      __syncwarp();
      if (kEpi == EPI_DELU_SUM) {
        const int col = lane & 15, r0 = (lane >> 4) * 16;
        float t = 0.f;
#pragma unroll
        for (int r = 0; r < 16; ++r) t += slab[(r0 + r) * 20 + col];
        t += __shfl_xor_sync(0xffffffffu, t, 16);
        if (lane < 16) wsum[warp * kMaxTileN + c + lane] = t;
      }
      if (cvec && ncol == 16) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int rr = 8 * i + (lane >> 2), qq = lane & 3;
          const int mr = m0 + warp * 32 + rr;
          if (mr < g.M)
            *reinterpret_cast<float4*>(cbase + (long long)mr * g.c_m + n0 + c + 4 * qq) =
                *reinterpret_cast<const float4*>(slab + rr * 20 + 4 * qq);
        }
      } else if (mrow) {
        for (int j = 0; j < ncol; ++j) cbase[(long long)m * g.c_m + n0 + c + j] = v[j];
      }
      __syncwarp();
    }
    if (kEpi == EPI_DELU_SUM) {
      __syncthreads();
      for (int n = tid; n < Nt && n0 + n < g.N; n += kMlpThreads)
        g.colsum[(long long)blockIdx.x * g.N + n0 + n] =
            ((wsum[n] + wsum[kMaxTileN + n]) + wsum[2 * kMaxTileN + n]) + wsum[3 * kMaxTileN + n];
    }
  } else if (nchunks == 0 && g.c_split) {
    // an empty split contributes zeros to the partial sums
    const int m = m0 + warp * 32 + lane;
    if (m < g.M) {
      float* crow = g.C + (long long)blockIdx.z * g.c_split + (long long)m * g.c_m;
      for (int n = n0; n < min(g.N, n0 + Nt); ++n) crow[n] = 0.f;
    }
  }
  if (!ok) {
    if (tid == 0 && g.err) atomicOr(g.err, DEVERR_TIMEOUT);
    // MMAs may still be in flight: wait (bounded) once more for the
    // outstanding commits before the tensor memory is released
    for (int b = 0; b < 2; ++b)
      if (waited[b] < issued[b]) mbar_wait(bar + b, (unsigned)waited[b] & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

// Sum of the split partial outputs in split order: C[m][n] = sum_s P[s][m][n].
__global__ void mlp_split_reduce_kernel(const float* __restrict__ P, int splits, long long split_len,
                                        float* __restrict__ C, long long n_total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_total;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += P[(long long)k * split_len + i];
    C[i] = s;
  }
}

}  // namespace

int mlp_tile_n(int M, int N, int K) {
  const int n16 = (N + 15) / 16 * 16;
  int nt = n16 < kMaxTileN ? n16 : kMaxTileN;
  const long long tiles = (long long)((M + kTileM - 1) / kTileM) * ((N + nt - 1) / nt);
  if ((K <= 32 || tiles < 2 * 152) && nt > 64) nt = 64;
  return nt;
}

size_t mlp_smem_bytes(int n_tile) {
  const size_t ab = (size_t)(kTileM + n_tile) * kChunkK * 4;   // one chunk of A and B
  return 2 * 2 * ab + kRawStages * ab + 64;
}

cudaError_t prepare_mlp_kernels() {
  const int smem = (int)mlp_smem_bytes(kMaxTileN);
  cudaError_t e = cudaFuncSetAttribute(mlp_gemm_kernel<EPI_PLAIN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_gemm_kernel<EPI_BIAS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_gemm_kernel<EPI_BIAS_ELU>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_gemm_kernel<EPI_DELU_SUM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_gemm_kernel<EPI_ELU>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

cudaError_t launch_mlp_gemm(const MlpGemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaSuccess;
  MlpGemmArgs g = a;
  if (g.n_tile <= 0) g.n_tile = mlp_tile_n(a.M, a.N, a.K);
  if (g.n_tile > kMaxTileN || g.n_tile % 16) return cudaErrorInvalidValue;
  const int splits = g.c_split ? (a.K + g.k_per_split - 1) / g.k_per_split : 1;
  if (!g.c_split) g.k_per_split = a.K;
  if (g.k_per_split <= 0) return cudaErrorInvalidValue;
  dim3 grid((a.M + kTileM - 1) / kTileM, (a.N + g.n_tile - 1) / g.n_tile, splits);
  const size_t smem = mlp_smem_bytes(g.n_tile);
  if (g.act_y && g.colsum) mlp_gemm_kernel<EPI_DELU_SUM><<<grid, kMlpThreads, smem, s>>>(g);
  else if (g.act_y || g.colsum) return cudaErrorInvalidValue;   // both or neither
  else if (g.bias && g.elu) mlp_gemm_kernel<EPI_BIAS_ELU><<<grid, kMlpThreads, smem, s>>>(g);
  else if (g.bias) mlp_gemm_kernel<EPI_BIAS><<<grid, kMlpThreads, smem, s>>>(g);
  else if (g.elu) mlp_gemm_kernel<EPI_ELU><<<grid, kMlpThreads, smem, s>>>(g);
  else mlp_gemm_kernel<EPI_PLAIN><<<grid, kMlpThreads, smem, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_mlp_split_reduce(const float* partial, int splits, long long split_len,
                                    float* C, long long n_total, cudaStream_t s) {
  long long blocks = (n_total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  mlp_split_reduce_kernel<<<(int)(blocks > 0 ? blocks : 1), 256, 0, s>>>(partial, splits,
                                                                        split_len, C, n_total);
  return cudaGetLastError();
}

cudaError_t launch_mlp_gemm_split(const MlpGemmArgs& a, float* work, long long work_floats,
                                  cudaStream_t s) {
  MlpGemmArgs g = a;
  const int n16 = (a.N + 15) / 16 * 16;
  const int nt = n16 < kMaxTileN ? n16 : kMaxTileN;   // long split products: the widest tile
  g.n_tile = nt;
  const long long tiles = (long long)((a.M + kTileM - 1) / kTileM) * ((a.N + nt - 1) / nt);
  int splits = 1;
  if (work && !a.bias && !a.elu && !a.act_y && !a.colsum && a.c_m == a.N && a.M > 0 && a.N > 0) {
    const long long want = (2 * 152 + tiles - 1) / tiles;   // about two CTAs per SM
    const long long chunks = (a.K + 31) / 32;
    long long sp = want < chunks ? want : chunks;
    const long long fit = work_floats / ((long long)a.M * a.N);
    if (sp > fit) sp = fit;
    splits = sp > 1 ? (int)sp : 1;
  }
  if (splits <= 1) {
    g.c_split = 0;
    return launch_mlp_gemm(g, s);
  }
  const long long chunks = (a.K + 31) / 32;
  g.k_per_split = (int)(((chunks + splits - 1) / splits) * 32);
  splits = (int)((a.K + g.k_per_split - 1) / g.k_per_split);
  g.C = work;
  g.c_split = (long long)a.M * a.N;
  cudaError_t e = launch_mlp_gemm(g, s);
  if (e != cudaSuccess) return e;
  return launch_mlp_split_reduce(work, splits, (long long)a.M * a.N, a.C, (long long)a.M * a.N, s);
}

}  // namespace sg

// ---- C ABI (include/sg_ppo.h) -------------------------------------------------
extern "C" sg_status sg_mlp_gemm(void* stream, const float* A, int64_t a_m, int64_t a_k,
                                 const float* B, int64_t b_n, int64_t b_k, const float* bias,
                                 int32_t elu, int32_t M, int32_t N, int32_t K, float* C,
                                 int64_t c_m, float* work, int64_t work_floats,
                                 int32_t split_tf32) {
  if (!A || !B || !C || M < 0 || N < 0 || K < 0 || work_floats < 0 || (work_floats > 0 && !work))
    return SG_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return SG_OK;
  static bool prepared = false;
  if (!prepared) {
    if (sg::prepare_mlp_kernels() != cudaSuccess) return SG_ERR_CUDA;
    prepared = true;
  }
  sg::MlpGemmArgs g{};
  g.A = A;
  g.a_m = a_m;
  g.a_k = a_k;
  g.B = B;
  g.b_n = b_n;
  g.b_k = b_k;
  g.C = C;
  g.c_m = c_m;
  g.bias = bias;
  g.M = M;
  g.N = N;
  g.K = K;
  g.elu = elu ? 1 : 0;
  g.split_tf32 = split_tf32 ? 1 : 0;
  return sg::launch_mlp_gemm_split(g, work, work_floats, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? SG_OK
             : SG_ERR_CUDA;
}
