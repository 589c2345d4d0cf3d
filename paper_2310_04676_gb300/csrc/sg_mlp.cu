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
// Split precision (3xTF32): x = hi + lo with hi = tf32(x) and lo = tf32(x - hi)
// (round to nearest);
// a b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b, the dropped lo_a lo_b term being
// about 2^-22 of a b, so the products carry FP32 accuracy with FP32
// accumulation (the published "3xTF32" emulation of FP32 matrix products).
//
// One CTA computes a 128 x Nt tile (Nt <= 128, a multiple of 16): eight
// warps copy, split and drain; lane 0 of a ninth warp issues the bulk copies
// of pre-split weights and the MMAs.  Raw FP32 operand chunks (16 wide in K)
// travel to shared memory by asynchronous copies two chunks ahead.  Each
// chunk of A is then split into its TF32 parts and stored in tensor memory
// (TMEM lane = row, one column per K value: the MMAs read A from there);
// each chunk of B is split into the tensor cores' K-major shared-memory
// layout without swizzle (8-row x 16-byte core matrices), or, for pre-split
// weights, arrives already split by bulk copies.  One CTA barrier per chunk;
// after it the issuing lane issues, per 8-wide K step, the three
// tcgen05.mma of kind::tf32 into an FP32 accumulator in tensor memory
// (column = n) and commits them to an mbarrier, while the eight warps split
// the next chunk; two operand stages alternate, a stage being refilled only
// after the mbarrier of the MMAs that read it has completed (bounded wait).
// The epilogue reads the accumulator with tcgen05.ld (warps w and w + 4
// share the TMEM lanes 32 (w % 4) .., taking alternate 16-column blocks),
// applies the epilogue and stores whole row segments.  Products with
// pre-split weights and at least two chunks run persistent CTAs (about two
// per SM) that take the output tiles in turn, the copies of a tile's first
// chunks overlapping the previous tile's epilogue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "sg.h"
#include "sg_internal.h"
#include "sg_mlp.h"

namespace sg {
namespace {

constexpr int kMlpThreads = 256;                  // threads that copy, split and drain
constexpr int kMlpBlock = kMlpThreads + 32;       // ... plus one warp that issues the MMAs
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          unsigned long long limit_ns) {
  if (mbar_poll(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 0; it < (1u << 24); ++it) {
    if (mbar_poll(bar, parity)) return true;
    if (gtimer() - t0 > limit_ns) return false;
  }
  return false;
}

// D (+)= A B^T with A (128 rows x 8 K, TF32) in tensor memory: row r in
// lane r, K value k in column a_tmem + k.
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                            uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate ? 1 : 0)
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

// Eight consecutive 32-bit columns of this thread's TMEM lane (warp w may
// address lanes 32 (w % 4) .. 32 (w % 4) + 31 only).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
      : "memory");
}

// ---- operand chunks ---------------------------------------------------------
// Rows [r0, r0 + nrows) x K [k0, k0 + 16) of X(r, k) = X[r xr + k xk] (zero
// outside R x K).  Raw chunks travel to shared memory by asynchronous
// 16-byte copies (cp.async, zero-filled outside the operand), kRawStages - 1
// chunks ahead.  When K is the contiguous direction (xk = 1) a 16-byte piece
// is four K values of one row -- one row of a core matrix -- and lands at its
// place in the tensor cores' layout, so the split into TF32 parts is an
// elementwise pass over the chunk.  When the rows are contiguous (xr = 1) a
// piece holds one K value of four rows: the chunk is kept K-major
// ([16][nrows]) and the split also transposes it (4-element units numbered
// core matrix by core matrix -- unit f has r = 8 (f >> 5) + (f & 7),
// kg = (f >> 3) & 3 -- so eight consecutive threads store the eight rows of
// one core matrix, conflict-free 16-byte stores).  Other strides are read by
// plain loads during the split.  Every thread's pieces are the same in each
// chunk, so their addresses are computed once (Loader) and advanced by one
// chunk per step.
constexpr int kRawStages = 3;
constexpr int kMaxTileN = 128;
constexpr int kUnits = kTileM * (kChunkK / 4) / kMlpThreads;   // 16-byte pieces per thread, <= 2

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
  else if (al && xr == 1 && (xk & 3) == 0 && (nrows & 15) == 0) o.layout = RAW_KMAJOR;
  return o;
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
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

// Per-thread copy state of one operand: up to kUnits 16-byte pieces per
// chunk, each with its source address at chunk 0, its byte offset in a raw
// stage and the bytes it holds (0: zero fill).  RAW_ROWS: piece j (u = tid +
// 256 j) is row r = 8 (u >> 5) + (u & 7), K group (u >> 3) & 3 (bytes shrink
// at the K tail); RAW_KMAJOR: piece j is K row k_j, rows 4 q .. 4 q + 3
// (q = tid % (nrows / 4)), stored at row position 4 q ^ kmajor_swz(k_j).
// In the K-major stage, row k holds its nrows values with the 8-row groups
// permuted by kmajor_swz(k) (an XOR of bits 3-4 of the row index), so that
// the split's reads -- 32 threads reading rows 8 w .. 8 w + 7 of the four K
// groups -- hit 32 different banks.
__device__ __forceinline__ int kmajor_swz(int k, int nrows) {
  return 8 * ((k >> 2) & ((nrows & 31) ? 1 : 3));
}
struct Loader {
  const float* src[kUnits];
  unsigned dst[kUnits];
  int bytes[kUnits];     // bytes of the piece inside the operand (rows / K range checks)
  int kofs[kUnits];      // K offset of the piece within a chunk
  int n;                 // pieces of this thread
};

__device__ __forceinline__ Loader make_loader(const Operand& o, int tid) {
  Loader L{};
  L.n = 0;
  if (o.layout == RAW_ROWS) {
#pragma unroll
    for (int j = 0; j < kUnits; ++j) {
      const int u = tid + j * kMlpThreads;
      if (u >= o.nrows * 4) break;
      // eight consecutive threads take the eight rows of one core matrix
      // (16-byte pieces 16 bytes apart: conflict-free shared-memory writes);
      // a warp still reads eight whole 64-byte row segments
      const int kg = (u >> 3) & 3;
      const int r = ((u >> 5) << 3) + (u & 7), gr = o.r0 + r;
      L.src[j] = gr < o.R ? o.X + (long long)gr * o.xr + 4 * kg : o.X;
      L.bytes[j] = gr < o.R ? 16 : 0;
      L.kofs[j] = 4 * kg;
      L.dst[j] = tile_off(r, 4 * kg);
      L.n = j + 1;
    }
  } else if (o.layout == RAW_KMAJOR) {
    const int rg = o.nrows >> 2;
#pragma unroll
    for (int j = 0; j < kUnits; ++j) {
      const int u = tid + j * kMlpThreads;
      if (u >= kChunkK * rg) break;
      const int k = u / rg, q = u - k * rg;
      const int gr = o.r0 + 4 * q;
      const int nr = max(0, min(4, o.R - gr));
      L.src[j] = nr ? o.X + (long long)k * o.xk + gr : o.X;
      L.bytes[j] = 4 * nr;
      L.kofs[j] = k;
      L.dst[j] = (unsigned)(k * o.nrows + ((4 * q) ^ kmajor_swz(k, o.nrows))) * 4u;
      L.n = j + 1;
    }
  }
  return L;
}

// Issue the copies of the chunk at K offset k0 into the raw stage at shared
// address `raw`.
__device__ __forceinline__ void raw_issue(const Operand& o, const Loader& L, int k0,
                                          unsigned raw) {
  const long long adv = (long long)k0 * o.xk;
  if (o.layout == RAW_ROWS) {
#pragma unroll
    for (int j = 0; j < kUnits; ++j) {
      if (j >= L.n) break;
      const int nk = max(0, min(4, o.K - (k0 + L.kofs[j])));
      const int b = L.bytes[j] ? 4 * nk : 0;
      cp_async16(raw + L.dst[j], b ? L.src[j] + adv : o.X, b);
    }
  } else if (o.layout == RAW_KMAJOR) {
#pragma unroll
    for (int j = 0; j < kUnits; ++j) {
      if (j >= L.n) break;
      const int b = k0 + L.kofs[j] < o.K ? L.bytes[j] : 0;
      cp_async16(raw + L.dst[j], b ? L.src[j] + adv : o.X, b);
    }
  }
}

// x rounded to the nearest TF32 value (10 mantissa bits), ties away from
// zero: half a unit of the last kept bit added to the magnitude bits, the 13
// dropped bits cleared.  For finite x below the largest TF32 value (a carry
// out of the exponent would give infinity).
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// TF32 parts: hi = round_tf32(x), lo = round_tf32(x - hi) (x - hi is exact in
// FP32), so x = hi + lo within 2^-22 |x|; the one-product mode needs hi only.
template <bool kSplit>
__device__ __forceinline__ void split4(const float (&v)[4], float4& h, float4& l) {
  h.x = round_tf32(v[0]);
  h.y = round_tf32(v[1]);
  h.z = round_tf32(v[2]);
  h.w = round_tf32(v[3]);
  if (kSplit) {
    l.x = round_tf32(v[0] - h.x);
    l.y = round_tf32(v[1] - h.y);
    l.z = round_tf32(v[2] - h.z);
    l.w = round_tf32(v[3] - h.w);
  }
}

// Split chunk k0 of B (from raw, or read directly for RAW_PLAIN) into the
// hi / lo shared-memory tiles the MMAs read (hi only in the one-product
// mode); used when B is not pre-split.
template <bool kSplit>
__device__ __forceinline__ void convert(const Operand& o, int k0, const float* raw, int tid,
                                        char* hi, char* lo) {
  const int units = o.nrows * (kChunkK / 4);
  if (o.layout == RAW_ROWS) {
    // the raw chunk is already in the tiles' layout: elementwise
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
      const int f = tid + u * kMlpThreads;
      if (f >= units) break;
      const float4 t = reinterpret_cast<const float4*>(raw)[f];
      const float v[4] = {t.x, t.y, t.z, t.w};
      float4 h, l;
      split4<kSplit>(v, h, l);
      reinterpret_cast<float4*>(hi)[f] = h;
      if (kSplit) reinterpret_cast<float4*>(lo)[f] = l;
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < kUnits; ++u) {
    const int f = tid + u * kMlpThreads;
    if (f >= units) break;
    const int r = ((f >> 5) << 3) + (f & 7), kg = (f >> 3) & 3;
    float v[4];
    if (o.layout == RAW_KMAJOR) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        v[j] = raw[(4 * kg + j) * o.nrows + (r ^ kmajor_swz(4 * kg + j, o.nrows))];
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
    split4<kSplit>(v, h, l);
    const unsigned off = tile_off(r, kg * 4);
    *reinterpret_cast<float4*>(hi + off) = h;
    if (kSplit) *reinterpret_cast<float4*>(lo + off) = l;
  }
}

// Split chunk k0 of A (128 rows: raw stage in the tiles' layout or K-major,
// or read directly for RAW_PLAIN) into its TF32 parts in tensor memory:
// warp w < 8 takes the rows of its TMEM lane quarter, 32 (w % 4) + lane, and
// the K values 8 (w / 4) .. 8 (w / 4) + 7 of the chunk; hi goes to columns
// t_hi + 8 (w / 4) .., lo to t_lo + 8 (w / 4) .. (hi only in the one-product
// mode).  The caller waits for the stores (tcgen05.wait::st).
template <bool kSplit>
__device__ __forceinline__ void split_a_tmem(const Operand& o, int k0, const char* raw, int warp,
                                             int lane, uint32_t t_hi, uint32_t t_lo) {
  const int lq = warp & 3, half = warp >> 2;
  const int r = lq * 32 + lane;
  float v[8];
  if (o.layout == RAW_ROWS) {
    const float4 a = *reinterpret_cast<const float4*>(raw + tile_off(r, 8 * half));
    const float4 b = *reinterpret_cast<const float4*>(raw + tile_off(r, 8 * half + 4));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
    v[4] = b.x;
    v[5] = b.y;
    v[6] = b.z;
    v[7] = b.w;
  } else if (o.layout == RAW_KMAJOR) {
    const float* rf = reinterpret_cast<const float*>(raw);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * half + j;
      v[j] = rf[k * o.nrows + (r ^ kmajor_swz(k, o.nrows))];
    }
  } else {
    const int gr = o.r0 + r;
    const float* row = o.X + (long long)gr * o.xr;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gk = k0 + 8 * half + j;
      v[j] = (gr < o.R && gk < o.K) ? __ldg(row + (long long)gk * o.xk) : 0.f;
    }
  }
  uint32_t h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float hf = round_tf32(v[j]);
    h[j] = __float_as_uint(hf);
    l[j] = kSplit ? __float_as_uint(round_tf32(v[j] - hf)) : 0u;
  }
  const uint32_t lane_base = (uint32_t)(lq * 32) << 16;
  tmem_st8(t_hi + lane_base + 8u * (uint32_t)half, h);
  if (kSplit) tmem_st8(t_lo + lane_base + 8u * (uint32_t)half, l);
}

// Epilogue modes (compile-time, no per-element branches): plain product,
// bias (+ ELU), ELU only, or the ELU derivative of the layer below with
// column sums.
enum EpiMode { EPI_PLAIN = 0, EPI_BIAS = 1, EPI_BIAS_ELU = 2, EPI_DELU_SUM = 3, EPI_ELU = 4 };

// ELU from the hardware exponential: e^x - 1 for x <= 0 (absolute error
// about 1e-7 against expm1; the layers' activations are O(1))
__device__ __forceinline__ float elu_fast(float x) { return x > 0.f ? x : __expf(x) - 1.f; }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Pre-split B operand (the weights, split once per weight update by
// mlp_presplit_kernel): chunk c, part p (0: hi, 1: lo) at
// b_pre + (2 c + p) npad 16, its npad rows in the tiles' layout (tile_off), so
// a CTA's Nt rows of one part are one contiguous block of Nt x 64 bytes and
// arrive by one bulk copy.
constexpr int kMmaBars = 3;     // MMA commits of chunk c signal barrier c % 3
// epilogue: per warp a 32 x 20-float slab, then [4][128] column partials
constexpr size_t kSlabBytes = (8 * 32 * 20 + 4 * 128) * sizeof(float);
constexpr int kPreStages = 3;   // pre-split B stages (chunk c in stage c % 3)

template <bool kPreB>
__host__ __device__ constexpr size_t smem_bytes_for(int n_tile) {
  // B tiles [kPreB ? 3 : 2][hi, lo]; raw A [3]; raw B [3] (not with kPreB);
  // the epilogue's slabs; 6 barriers, the TMEM address and the abort flag
  // (A's split parts live in tensor memory)
  return (size_t)kRawStages * kTileM * kChunkK * 4 +
         (size_t)(kPreB ? 2 * kPreStages : 2 * 2 + kRawStages) * n_tile * kChunkK * 4 +
         kSlabBytes + 64;
}

template <int kEpi, bool kPreB, bool kSplit>
__global__ void __launch_bounds__(kMlpBlock, 2) mlp_gemm_kernel(MlpGemmArgs g) {
  extern __shared__ __align__(1024) char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // warps 0-7 copy and split the operands and drain the accumulator; lane 0
  // of warp 8 alone issues the pre-split B copies, the MMAs and their commits
  const bool conv = tid < kMlpThreads, issuer = tid == kMlpThreads;
  const unsigned long long lim = g.wait_ns ? g.wait_ns : kMmaWaitNs;   // bound of every wait
  const int Nt = g.n_tile;                         // multiple of 16, <= 128
  // output tiles, row-major (consecutive tiles share A's rows); this CTA
  // takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
  const int tiles_n = (g.N + Nt - 1) / Nt;
  const int ntiles = ((g.M + kTileM - 1) / kTileM) * tiles_n;
  const int kbeg = blockIdx.z * g.k_per_split;
  const int kend = min(g.K, kbeg + g.k_per_split);
  const int a_part = kTileM * kChunkK * 4, b_part = Nt * kChunkK * 4;
  char* const b_tiles = sm;
  char* const raw_a = b_tiles + (kPreB ? kPreStages : 2) * 2 * b_part;
  char* const raw_b = raw_a + kRawStages * a_part;
  char* const slabs = raw_b + (kPreB ? 0 : kRawStages * b_part);
  uint64_t* const bars = reinterpret_cast<uint64_t*>(slabs + kSlabBytes);   // [3] MMA, [3] B
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bars + 6);
  volatile int* const abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // tensor memory: the accumulator in columns 0 .. Nt - 1, then A's split
  // parts, stage s: hi at a_col0 + 32 s, lo 16 columns further
  const uint32_t a_col0 = Nt <= 64 ? 64u : 128u;
  const uint32_t ncols = Nt <= 64 ? 128u : 256u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 6; ++b) mbar_init1(bars + b);
    *abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(kTileM, Nt);

  const int nchunks = kbeg < kend ? (kend - kbeg + kChunkK - 1) / kChunkK : 0;
  auto tile_m0 = [&](int t) { return (t / tiles_n) * kTileM; };
  auto tile_n0 = [&](int t) { return (t % tiles_n) * Nt; };
  int tile = blockIdx.x;
  // the chunk pipeline runs across this CTA's tiles (chunk G of the CTA's
  // stream: stage G & 1, raw stage G % 3, barriers G % 3): the copies of the
  // next tile's first two chunks start during the current tile's last two,
  // and so overlap its epilogue.  A tile boundary is crossed at most once by
  // a two-chunk lookahead only with two or more chunks per tile; shorter
  // products take one tile per CTA (the launcher's grid).
  int nxt = tile + (int)gridDim.x;
  bool has_next = kPreB && nxt < ntiles && nchunks >= 2;   // the launcher's persistent grids
  Operand opa = make_operand(g.A, g.a_m, g.a_k, g.M, g.K, tile_m0(tile), kTileM);
  const Operand opb = make_operand(g.B, g.b_n, g.b_k, g.N, g.K, tile_n0(tile), Nt);
  Loader la{}, lb{};
  if (conv) la = make_loader(opa, tid);
  if (!kPreB && conv) lb = make_loader(opb, tid);
  Operand opa_n = opa;
  Loader la_n = la;
  if (has_next) {
    opa_n = make_operand(g.A, g.a_m, g.a_k, g.M, g.K, tile_m0(nxt), kTileM);
    if (conv) la_n = make_loader(opa_n, tid);
  }
  const unsigned raw_a_s = smem_addr(raw_a), raw_b_s = smem_addr(raw_b);
  // the issuer's account of the pre-split B copies and of the MMA commits
  int b_issued = 0, b_waited = 0, committed = 0;
  // B of stream chunk G: chunk c of the tile at column n0x
  auto issue_pre_b = [&](int G, int n0x, int c) {
    if (g.fault && G == 0) {
      // test hook: the copy of the stream's first weight chunk is left out
      // (but counted, so that an abort waits for every later copy)
      ++b_issued;
      return;
    }
    uint64_t* full = bars + kMmaBars + G % kPreStages;
    char* dst = b_tiles + (G % kPreStages) * 2 * b_part;
    const float* src = g.b_pre + (long long)(kbeg / kChunkK + c) * 2 * g.b_npad * kChunkK +
                       (long long)n0x * kChunkK;
    mbar_expect_tx(full, 2u * b_part);
    bulk_copy(dst, src, b_part, full);
    bulk_copy(dst + b_part, src + (long long)g.b_npad * kChunkK, b_part, full);
    ++b_issued;
  };

  bool ok = true;
  // prologue: the raw copies of chunks 0 and 1 and the pre-split B of chunk 0
  // in flight; chunk 0 landed before the loop starts
#pragma unroll
  for (int c = 0; c < kRawStages - 1; ++c) {
    if (c < nchunks) {
      raw_issue(opa, la, kbeg + c * kChunkK, raw_a_s + c * a_part);
      if (!kPreB) raw_issue(opb, lb, kbeg + c * kChunkK, raw_b_s + c * b_part);
    }
    cp_async_commit();
  }
  if (kPreB && issuer && nchunks > 0) issue_pre_b(0, tile_n0(tile), 0);
  cp_async_wait<kRawStages - 2>();
  __syncthreads();
  int G0 = 0;                                     // stream index of the tile's chunk 0
  for (;;) {
    const int m0 = tile_m0(tile), n0 = tile_n0(tile);
    // One CTA barrier per chunk: after it, chunk c's tiles are split (warps
    // 0-7) and chunk c + 1's raw copies have landed; the issuer then issues
    // chunk c's MMAs while the other warps go on to split chunk c + 1.
    for (int c = 0; c < nchunks; ++c) {
      const int G = G0 + c, ts = G & 1, rs = G % kRawStages;
      {
        // the raw stage of chunk G + 2 held chunk G - 1, split before the last barrier
        const int cn = c + kRawStages - 1, Gn = G + kRawStages - 1;
        if (cn < nchunks) {
          raw_issue(opa, la, kbeg + cn * kChunkK, raw_a_s + (Gn % kRawStages) * a_part);
          if (!kPreB)
            raw_issue(opb, lb, kbeg + cn * kChunkK, raw_b_s + (Gn % kRawStages) * b_part);
        } else if (has_next) {
          raw_issue(opa_n, la_n, kbeg + (cn - nchunks) * kChunkK,
                    raw_a_s + (Gn % kRawStages) * a_part);
        }
        cp_async_commit();
      }
      // stage ts (A's tensor-memory columns, B's split tiles) and the B stage
      // of chunk G + 1 were read by the MMAs of chunk G - 2
      if (G >= 2 &&
          !mbar_wait(bars + (G - 2) % kMmaBars, (unsigned)((G - 2) / kMmaBars) & 1u, lim))
        *abort_flag = 1;
      if (kPreB && issuer) {
        if (c + 1 < nchunks) issue_pre_b(G + 1, n0, c + 1);
        else if (has_next) issue_pre_b(G + 1, tile_n0(nxt), 0);
      }
      const uint32_t a_hi = tmem + a_col0 + 32u * (uint32_t)ts;
      char* const bhi = b_tiles + (kPreB ? G % kPreStages : ts) * 2 * b_part;
      if (conv) {
        // after the wait above: the MMAs of chunk G - 2 no longer read the stage
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        split_a_tmem<kSplit>(opa, kbeg + c * kChunkK, raw_a + rs * a_part, warp, lane, a_hi,
                             a_hi + 16u);
        if (!kPreB)
          convert<kSplit>(opb, kbeg + c * kChunkK,
                          reinterpret_cast<const float*>(raw_b + rs * b_part), tid, bhi,
                          bhi + b_part);
      }
      // B's split tiles (written by these threads) are read by the MMAs
      if (!kPreB) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      cp_async_wait<kRawStages - 2>();            // this thread's copies of chunk G + 1 landed
      if (conv) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (*abort_flag) {
        ok = false;
        break;
      }
      if (issuer) {
        bool bok = true;
        if (kPreB) {
          bok = mbar_wait(bars + kMmaBars + G % kPreStages, (unsigned)(G / kPreStages) & 1u, lim);
          if (bok) ++b_waited;
        }
        if (bok) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int ks = 0; ks < kChunkK / 8; ++ks) {
            const unsigned koff = (unsigned)ks * 2 * kLbo;   // two core matrices per K step
            const uint32_t ah = a_hi + 8u * (uint32_t)ks;    // eight TMEM columns per K step
            const uint32_t al = ah + 16u;
            const uint64_t bh = smem_desc(smem_addr(bhi) + koff);
            const uint64_t bl = smem_desc(smem_addr(bhi + b_part) + koff);
            mma_tf32_ta(tmem, ah, bh, idesc, c > 0 || ks > 0);
            if (kSplit) {
              mma_tf32_ta(tmem, ah, bl, idesc, true);
              mma_tf32_ta(tmem, al, bh, idesc, true);
            }
          }
          mma_commit(bars + G % kMmaBars);
          ++committed;
        } else {
          *abort_flag = 1;
        }
      }
    }
    if (!ok) break;
    G0 += nchunks;
    // the tile's accumulator is complete once its last chunk's commit is
    if (nchunks > 0)
      ok = __syncthreads_and(
          mbar_wait(bars + (G0 - 1) % kMmaBars, (unsigned)((G0 - 1) / kMmaBars) & 1u, lim));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) break;

    if (nchunks > 0) {
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its rows m0 + 32 (w % 4)
      // + lane) and the 16-column blocks of parity w / 4.  Per block each
      // thread finishes its row's values (bias, ELU, or the ELU derivative of
      // the layer below) and parks them in a shared-memory slab of the warp
      // (row pitch 20 floats, a region of its own).  From the slab the warp
      // sums the columns (lane l: column l % 16 over 16 rows, then the two
      // halves; fixed order) into the partials of its lane quarter, and
      // stores whole 64-byte row segments, four lanes per row, eight rows
      // per instruction (scalar stores at ragged edges or unaligned
      // outputs).  After the last block the four lane quarters' partials are
      // added in order (per 128-row tile of the output).
      const int lq = warp & 3, half = warp >> 2;
      const int m = m0 + lq * 32 + lane;
      const bool mrow = m < g.M;
      float* cbase = g.C + (long long)blockIdx.z * g.c_split;
      float* slab = reinterpret_cast<float*>(slabs) + warp * 32 * 20;
      float* wsum = reinterpret_cast<float*>(slabs) + 8 * 32 * 20;       // [4][128]
      const bool cvec = (g.c_m & 3) == 0 && (reinterpret_cast<uintptr_t>(cbase) & 15) == 0;
      const bool yvec = kEpi == EPI_DELU_SUM && (g.c_m & 3) == 0 &&
                        (reinterpret_cast<uintptr_t>(g.act_y) & 15) == 0;
      const bool bvec = (reinterpret_cast<uintptr_t>(g.bias + n0) & 15) == 0;
      for (int c = 16 * half; conv && c < Nt; c += 32) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)c, v);
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
          if (ncol == 16 && bvec) {
  #pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 t = __ldg(reinterpret_cast<const float4*>(g.bias + n0 + c) + q);
              v[4 * q] += t.x;
              v[4 * q + 1] += t.y;
              v[4 * q + 2] += t.z;
              v[4 * q + 3] += t.w;
            }
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
          if (lane < 16) wsum[lq * kMaxTileN + c + lane] = t;
        }
        if (cvec && ncol == 16) {
  #pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int rr = 8 * i + (lane >> 2), qq = lane & 3;
            const int mr = m0 + lq * 32 + rr;
            if (mr < g.M)
              *reinterpret_cast<float4*>(cbase + (long long)mr * g.c_m + n0 + c + 4 * qq) =
                  *reinterpret_cast<const float4*>(slab + rr * 20 + 4 * qq);
          }
        } else if (mrow) {
  #pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j < ncol) cbase[(long long)m * g.c_m + n0 + c + j] = v[j];
        }
        __syncwarp();
      }
      if (kEpi == EPI_DELU_SUM) {
        __syncthreads();
        for (int n = tid; n < Nt && n0 + n < g.N; n += kMlpThreads)
          g.colsum[(long long)(m0 / kTileM) * g.N + n0 + n] =
              ((wsum[n] + wsum[kMaxTileN + n]) + wsum[2 * kMaxTileN + n]) + wsum[3 * kMaxTileN + n];
      }
    } else if (g.c_split) {
      // an empty split contributes zeros to the partial sums: thread t takes
      // row m0 + t % 128 and every other column from n0 + t / 128
      const int m = m0 + (tid & (kTileM - 1));
      if (conv && m < g.M) {
        float* crow = g.C + (long long)blockIdx.z * g.c_split + (long long)m * g.c_m;
        for (int n = n0 + tid / kTileM; n < min(g.N, n0 + Nt); n += kMlpThreads / kTileM)
          crow[n] = 0.f;
      }
    }
    if (!has_next) break;
    // the next tile's MMAs overwrite the accumulator: every thread done
    // reading it (and with the slabs) first
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tile = nxt;
    opa = opa_n;
    la = la_n;
    nxt = tile + (int)gridDim.x;
    has_next = kPreB && nxt < ntiles;
    if (has_next) {
      opa_n = make_operand(g.A, g.a_m, g.a_k, g.M, g.K, tile_m0(nxt), kTileM);
      if (conv) la_n = make_loader(opa_n, tid);
    }
  }
  cp_async_wait<0>();
  if (!ok) {
    if (issuer) {
      if (g.err) atomicOr(g.err, DEVERR_TIMEOUT);
      // copies and MMAs may still be in flight: wait (bounded) for the
      // outstanding B copies and the last commit before the shared and
      // tensor memory are released
      for (int j = b_waited; j < b_issued; ++j)
        mbar_wait(bars + kMmaBars + j % kPreStages, (unsigned)(j / kPreStages) & 1u, lim);
      if (committed > 0)
        mbar_wait(bars + (committed - 1) % kMmaBars, (unsigned)((committed - 1) / kMmaBars) & 1u,
                  lim);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

// Sum of the split partial outputs in a fixed order: C[i] = sum_s P[s][i],
// warp w of a block adding the splits s = w, w + 8, ... in increasing order
// for 32 consecutive outputs (four floats per lane when kVec), then the
// eight warp sums added in warp order.
template <bool kVec>
__global__ void __launch_bounds__(256) mlp_split_reduce_kernel(const float* __restrict__ P,
                                                               int splits, long long split_len,
                                                               float* __restrict__ C,
                                                               long long n_total) {
  using T = typename std::conditional<kVec, float4, float>::type;
  __shared__ T sh[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n = kVec ? n_total / 4 : n_total, len = kVec ? split_len / 4 : split_len;
  const T* p = reinterpret_cast<const T*>(P);
  T* c = reinterpret_cast<T*>(C);
  auto add = [](T& a, const T& b) {
    if constexpr (kVec) {
      a.x += b.x;
      a.y += b.y;
      a.z += b.z;
      a.w += b.w;
    } else {
      a += b;
    }
  };
  for (long long base = blockIdx.x * 32LL; base < n; base += gridDim.x * 32LL) {
    const long long i = base + lane;
    T acc{};
    if (i < n) {
#pragma unroll 4
      for (int s = warp; s < splits; s += 8) add(acc, __ldg(p + (long long)s * len + i));
    }
    sh[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && i < n) {
      T t = sh[0][lane];
#pragma unroll
      for (int w = 1; w < 8; ++w) add(t, sh[w][lane]);
      c[i] = t;
    }
    __syncthreads();
  }
}

// Split W (B(n, k) = W[n wn + k wk], N x K) into the pre-split layout above:
// dst[(2 c + p) npad 16 + e], e the float index of (n, k - 16 c) in the tiles'
// layout; parts beyond N x K are zero; lo = 0 in the one-product mode.
__global__ void mlp_presplit_kernel(PresplitJobs jobs, int split_tf32) {
  long long base = 0;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int j = 0; j < jobs.n; ++j) {
    const PresplitJob& J = jobs.job[j];
    const long long chunk = 2LL * J.npad * kChunkK;
    const long long count = (long long)((J.K + kChunkK - 1) / kChunkK) * chunk;
    long long i = i0 - base;
    if (i < 0) i += (-i + stride - 1) / stride * stride;
    for (; i < count; i += stride) {
      const int c = (int)(i / chunk);
      const long long rem = i - (long long)c * chunk;
      const int p = (int)(rem / ((long long)J.npad * kChunkK));
      const int e = (int)(rem - (long long)p * J.npad * kChunkK);
      // e -> (n, kk): 128 floats per 8-row group, 32 per K group, 4 per row
      const int n8 = e >> 7, w = e & 127, kg = w >> 5, w2 = w & 31;
      const int n = n8 * 8 + (w2 >> 2), k = c * kChunkK + kg * 4 + (w2 & 3);
      const float x = (n < J.N && k < J.K) ? J.W[(long long)n * J.wn + (long long)k * J.wk] : 0.f;
      const float hi = round_tf32(x);
      J.dst[i] = p == 0 ? hi : (split_tf32 ? round_tf32(x - hi) : 0.f);
    }
    base += count;
  }
}

// ---- narrow products on the FP32 pipes ---------------------------------------
// Products with a short inner dimension and few outputs per row (the input
// gradient below an 8- or 1-wide output layer: K * N <= 2048) or an output of
// at most 16 columns (the output layers) do a few FMAs per element they move:
// a 128-row tensor-core tile is set up, filled and drained for one or two
// chunks of work.  They run as plain FP32 FMA loops instead (exact FP32
// products, accumulated in a fixed order), their operand rows staged in
// shared memory by coalesced loads.
constexpr int kNarrowRows = 128;      // rows per block (the bias-gradient partials' tile)
constexpr int kNarrowMaxK = 32;

__device__ __forceinline__ bool al16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// C[m][n] = epi(sum_{k < K} A[m a_m + k] B(n, k)), K <= 32, N <= 256.  Block:
// 128 rows; warp w takes column strip w % S (S = ceil(N / 32)) and the rows
// r = w / S (mod P = 8 / S) of them, lane l column 32 (w % S) + l with its K
// weights in registers; A's rows broadcast from shared memory.  The input-
// gradient epilogue also writes the block's column sums (fixed order: rows in
// order per thread, then the P row classes in order).
template <int kEpi>
__global__ void __launch_bounds__(256) narrow_k_kernel(MlpGemmArgs g) {
  __shared__ __align__(16) float As[kNarrowRows * kNarrowMaxK];
  __shared__ float csum[8][256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = g.K, N = g.N, K4 = (K + 3) & ~3;
  const int m0 = blockIdx.x * kNarrowRows;
  // stage A's rows [128][K4] (zero beyond M x K)
  if (al16(g.A) && (g.a_m & 3) == 0 && (K & 3) == 0) {
    const int q4 = K4 >> 2;
    for (int u = tid; u < kNarrowRows * q4; u += 256) {
      const int r = u / q4, q = u - r * q4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m0 + r < g.M) v = __ldg(reinterpret_cast<const float4*>(g.A + (long long)(m0 + r) * g.a_m) + q);
      reinterpret_cast<float4*>(As)[r * q4 + q] = v;
    }
  } else {
    for (int u = tid; u < kNarrowRows * K4; u += 256) {
      const int r = u / K4, k = u - r * K4;
      As[u] = (m0 + r < g.M && k < K) ? __ldg(g.A + (long long)(m0 + r) * g.a_m + k) : 0.f;
    }
  }
  __syncthreads();
  const int S = (N + 31) / 32, P = S >= 8 ? 1 : 8 / S;
  for (int job = warp; job < S * P; job += 8) {
    const int strip = job % S, phase = job / S;
    const int n = strip * 32 + lane;
    const bool nv = n < N;
    float w[kNarrowMaxK];
#pragma unroll
    for (int k = 0; k < kNarrowMaxK; ++k)
      w[k] = (nv && k < K) ? __ldg(g.B + (long long)n * g.b_n + (long long)k * g.b_k) : 0.f;
    const float bn = ((kEpi == EPI_BIAS || kEpi == EPI_BIAS_ELU) && nv) ? __ldg(g.bias + n) : 0.f;
    float cs = 0.f;
    // rows phase, phase + P, ... in order, four at a time so that the four
    // rows' activation loads are in flight together
    const int nrows = min(kNarrowRows, g.M - m0);
    constexpr int kU = 4;
    for (int r0 = phase; r0 < nrows; r0 += kU * P) {
      float y[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int r = r0 + u * P;
        y[u] = (kEpi == EPI_DELU_SUM && nv && r < nrows)
                   ? __ldg(g.act_y + (long long)(m0 + r) * g.c_m + n)
                   : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int r = r0 + u * P;
        if (r >= nrows) break;
        const float4* x4 = reinterpret_cast<const float4*>(As + r * K4);
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < kNarrowMaxK / 4; ++q) {
          if (4 * q >= K4) break;
          const float4 x = x4[q];
          acc = fmaf(x.x, w[4 * q], acc);
          acc = fmaf(x.y, w[4 * q + 1], acc);
          acc = fmaf(x.z, w[4 * q + 2], acc);
          acc = fmaf(x.w, w[4 * q + 3], acc);
        }
        if (kEpi == EPI_BIAS || kEpi == EPI_BIAS_ELU) acc += bn;
        if (kEpi == EPI_BIAS_ELU || kEpi == EPI_ELU) acc = elu_fast(acc);
        if (kEpi == EPI_DELU_SUM) {
          acc *= y[u] > 0.f ? 1.f : y[u] + 1.f;
          cs += nv ? acc : 0.f;
        }
        if (nv) g.C[(long long)(m0 + r) * g.c_m + n] = acc;
      }
    }
    if (kEpi == EPI_DELU_SUM && nv) csum[phase][n] = cs;
  }
  if (kEpi == EPI_DELU_SUM) {
    __syncthreads();
    for (int n = tid; n < N; n += 256) {
      float t = 0.f;
      for (int ph = 0; ph < P; ++ph) t += csum[ph][n];
      g.colsum[(long long)blockIdx.x * N + n] = t;
    }
  }
}

// C[m][n] = epi(sum_k A[m a_m + k] B(n, k)), N <= 16, K <= 64 (a multiple of
// 4): thread t of 128 takes row m0 + t with its N sums in registers; A's rows
// staged with a pitch of K + 4 floats (conflict-free 16-byte reads), B in
// shared memory (broadcast reads).
constexpr int kNarrowMaxN = 16, kNarrowNMaxK = 64;
template <int kEpi>
__global__ void __launch_bounds__(128) narrow_n_kernel(MlpGemmArgs g) {
  __shared__ __align__(16) float As[kNarrowRows * (kNarrowNMaxK + 4)];
  __shared__ __align__(16) float Ws[kNarrowMaxN * kNarrowNMaxK];
  const int tid = threadIdx.x;
  const int K = g.K, N = g.N, q4 = K >> 2, pitch = K + 4;
  const int m0 = blockIdx.x * kNarrowRows;
  for (int u = tid; u < kNarrowRows * q4; u += kNarrowRows) {
    const int r = u / q4, q = u - r * q4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m0 + r < g.M) v = __ldg(reinterpret_cast<const float4*>(g.A + (long long)(m0 + r) * g.a_m) + q);
    *reinterpret_cast<float4*>(As + r * pitch + 4 * q) = v;
  }
  for (int u = tid; u < kNarrowMaxN * K; u += kNarrowRows) {
    const int n = u / K, k = u - n * K;
    Ws[u] = n < N ? __ldg(g.B + (long long)n * g.b_n + (long long)k * g.b_k) : 0.f;
  }
  __syncthreads();
  const int m = m0 + tid;
  if (m >= g.M) return;
  float acc[kNarrowMaxN];
#pragma unroll
  for (int n = 0; n < kNarrowMaxN; ++n) acc[n] = 0.f;
  for (int q = 0; q < q4; ++q) {
    const float4 x = *reinterpret_cast<const float4*>(As + tid * pitch + 4 * q);
#pragma unroll
    for (int n = 0; n < kNarrowMaxN; ++n) {
      if (n >= N) break;
      const float4 w = *reinterpret_cast<const float4*>(Ws + n * K + 4 * q);
      acc[n] = fmaf(x.x, w.x, acc[n]);
      acc[n] = fmaf(x.y, w.y, acc[n]);
      acc[n] = fmaf(x.z, w.z, acc[n]);
      acc[n] = fmaf(x.w, w.w, acc[n]);
    }
  }
#pragma unroll
  for (int n = 0; n < kNarrowMaxN; ++n) {
    if (n >= N) break;
    float v = acc[n];
    if (kEpi == EPI_BIAS || kEpi == EPI_BIAS_ELU) v += __ldg(g.bias + n);
    if (kEpi == EPI_BIAS_ELU || kEpi == EPI_ELU) v = elu_fast(v);
    g.C[(long long)m * g.c_m + n] = v;
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

size_t mlp_smem_bytes(int n_tile, bool pre_b) {
  return pre_b ? smem_bytes_for<true>(n_tile) : smem_bytes_for<false>(n_tile);
}

namespace {
template <int kEpi, bool kPreB, bool kSplit>
cudaError_t allow_smem() {
  return cudaFuncSetAttribute(mlp_gemm_kernel<kEpi, kPreB, kSplit>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes_for<kPreB>(kMaxTileN));
}
template <bool kPreB, bool kSplit>
cudaError_t allow_smem_all() {
  cudaError_t e = allow_smem<EPI_PLAIN, kPreB, kSplit>();
  if (e == cudaSuccess) e = allow_smem<EPI_BIAS, kPreB, kSplit>();
  if (e == cudaSuccess) e = allow_smem<EPI_BIAS_ELU, kPreB, kSplit>();
  if (e == cudaSuccess) e = allow_smem<EPI_DELU_SUM, kPreB, kSplit>();
  if (e == cudaSuccess) e = allow_smem<EPI_ELU, kPreB, kSplit>();
  return e;
}
template <bool kPreB, bool kSplit>
void launch_epi2(const MlpGemmArgs& g, dim3 grid, size_t smem, cudaStream_t s) {
  if (g.act_y) mlp_gemm_kernel<EPI_DELU_SUM, kPreB, kSplit><<<grid, kMlpBlock, smem, s>>>(g);
  else if (g.bias && g.elu)
    mlp_gemm_kernel<EPI_BIAS_ELU, kPreB, kSplit><<<grid, kMlpBlock, smem, s>>>(g);
  else if (g.bias) mlp_gemm_kernel<EPI_BIAS, kPreB, kSplit><<<grid, kMlpBlock, smem, s>>>(g);
  else if (g.elu) mlp_gemm_kernel<EPI_ELU, kPreB, kSplit><<<grid, kMlpBlock, smem, s>>>(g);
  else mlp_gemm_kernel<EPI_PLAIN, kPreB, kSplit><<<grid, kMlpBlock, smem, s>>>(g);
}
template <bool kPreB>
void launch_epi(const MlpGemmArgs& g, dim3 grid, size_t smem, cudaStream_t s) {
  if (g.split_tf32) launch_epi2<kPreB, true>(g, grid, smem, s);
  else launch_epi2<kPreB, false>(g, grid, smem, s);
}
}  // namespace

cudaError_t prepare_mlp_kernels() {
  cudaError_t e = allow_smem_all<false, true>();
  if (e == cudaSuccess) e = allow_smem_all<true, true>();
  if (e == cudaSuccess) e = allow_smem_all<false, false>();
  if (e == cudaSuccess) e = allow_smem_all<true, false>();
  return e;
}

int presplit_npad(int N) { return (N + kMaxTileN - 1) / kMaxTileN * kMaxTileN; }

long long presplit_floats(int N, int K) {
  return (long long)((K + kChunkK - 1) / kChunkK) * 2 * presplit_npad(N) * kChunkK;
}

cudaError_t launch_mlp_presplit(const PresplitJobs& jobs, int split_tf32, cudaStream_t s) {
  if (jobs.n < 0 || jobs.n > kMaxPresplitJobs) return cudaErrorInvalidValue;
  long long total = 0;
  for (int j = 0; j < jobs.n; ++j) {
    const PresplitJob& J = jobs.job[j];
    if (!J.W || !J.dst || J.N <= 0 || J.K <= 0 || J.npad != presplit_npad(J.N) ||
        (reinterpret_cast<uintptr_t>(J.dst) & 15))
      return cudaErrorInvalidValue;
    total += presplit_floats(J.N, J.K);
  }
  if (total == 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  mlp_presplit_kernel<<<(int)blocks, 256, 0, s>>>(jobs, split_tf32);
  return cudaGetLastError();
}

int mlp_narrow_kind(const MlpGemmArgs& g) {
  if (!g.narrow || g.M <= 0 || g.N <= 0 || g.K <= 0 || g.c_split) return NARROW_NONE;
  if (g.a_k != 1) return NARROW_NONE;
  // a few FMAs per row: below that the tensor-core tile's setup and drain
  // dominate, above it the FMA loops do
  if (g.K <= kNarrowMaxK && g.N <= 256 && g.K * g.N <= 2048) return NARROW_K;
  if (g.N <= kNarrowMaxN && g.K <= kNarrowNMaxK && (g.K & 3) == 0 && (g.a_m & 3) == 0 &&
      (reinterpret_cast<uintptr_t>(g.A) & 15) == 0 && !g.act_y && !g.colsum)
    return NARROW_N;
  return NARROW_NONE;
}

namespace {
template <int kEpi>
void launch_narrow_rows(const MlpGemmArgs& g, int kind, cudaStream_t s) {
  const int blocks = (g.M + kNarrowRows - 1) / kNarrowRows;
  if (kind == NARROW_K) narrow_k_kernel<kEpi><<<blocks, 256, 0, s>>>(g);
  else narrow_n_kernel<kEpi><<<blocks, kNarrowRows, 0, s>>>(g);
}

// the row kinds (forward and input gradient): one launch
cudaError_t launch_narrow(const MlpGemmArgs& g, int kind, cudaStream_t s) {
  if (g.act_y) launch_narrow_rows<EPI_DELU_SUM>(g, kind, s);
  else if (g.bias && g.elu) launch_narrow_rows<EPI_BIAS_ELU>(g, kind, s);
  else if (g.bias) launch_narrow_rows<EPI_BIAS>(g, kind, s);
  else if (g.elu) launch_narrow_rows<EPI_ELU>(g, kind, s);
  else launch_narrow_rows<EPI_PLAIN>(g, kind, s);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_mlp_gemm(const MlpGemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaSuccess;
  if (!a.act_y != !a.colsum) return cudaErrorInvalidValue;   // both or neither
  const int nk = mlp_narrow_kind(a);
  if (nk == NARROW_K || nk == NARROW_N) return launch_narrow(a, nk, s);
  MlpGemmArgs g = a;
  if (g.n_tile <= 0) g.n_tile = mlp_tile_n(a.M, a.N, a.K);
  if (g.n_tile > kMaxTileN || g.n_tile % 16) return cudaErrorInvalidValue;
  const int splits = g.c_split ? (a.K + g.k_per_split - 1) / g.k_per_split : 1;
  if (!g.c_split) g.k_per_split = a.K;
  if (g.k_per_split <= 0) return cudaErrorInvalidValue;
  const bool pre = g.b_pre != nullptr;
  if (pre) {
    // the CTAs' row blocks must lie inside the pre-split rows, the copies
    // 16-byte aligned, and the K splits start at whole chunks
    const int ntiles = (a.N + g.n_tile - 1) / g.n_tile;
    if (g.b_npad != presplit_npad(a.N) || ntiles * g.n_tile > g.b_npad ||
        (reinterpret_cast<uintptr_t>(g.b_pre) & 15) || (splits > 1 && g.k_per_split % kChunkK))
      return cudaErrorInvalidValue;
  }
  // tiles in one dimension; products with pre-split weights and two or more
  // chunks per tile run persistent CTAs (about two per SM) that take the
  // tiles in turn, the others one CTA per tile
  const long long ntiles =
      (long long)((a.M + kTileM - 1) / kTileM) * ((a.N + g.n_tile - 1) / g.n_tile);
  const int kchunks = (g.k_per_split + kChunkK - 1) / kChunkK;
  const long long ctas = (pre && splits == 1 && kchunks >= 2) ? std::min<long long>(ntiles, 2 * 152)
                                                             : ntiles;
  if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)ctas, 1, splits);
  const size_t smem = mlp_smem_bytes(g.n_tile, pre);
  if (pre) launch_epi<true>(g, grid, smem, s);
  else launch_epi<false>(g, grid, smem, s);
  return cudaGetLastError();
}

cudaError_t launch_mlp_split_reduce(const float* partial, int splits, long long split_len,
                                    float* C, long long n_total, cudaStream_t s) {
  const bool vec = (split_len & 3) == 0 && (n_total & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(partial) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(C) & 15) == 0;
  const long long n = vec ? n_total / 4 : n_total;
  long long blocks = (n + 31) / 32;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  if (vec)
    mlp_split_reduce_kernel<true><<<(int)blocks, 256, 0, s>>>(partial, splits, split_len, C, n_total);
  else
    mlp_split_reduce_kernel<false><<<(int)blocks, 256, 0, s>>>(partial, splits, split_len, C,
                                                               n_total);
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
    g.n_tile = 0;
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
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
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
  g.narrow = split_tf32 == 2 ? 1 : 0;
  // a product with enough row tiles to fill the GPU and a work buffer that
  // holds B's TF32 parts: split B once, then every CTA copies its parts
  const int nk = sg::mlp_narrow_kind(g);
  if (nk == sg::NARROW_K || nk == sg::NARROW_N)
    return sg::launch_mlp_gemm(g, s) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
  const long long tiles = (long long)((M + 127) / 128) * ((N + 127) / 128);
  const bool k_split = !bias && !elu && c_m == N && tiles < 2 * 152 && K > 32;
  if (work && K > 0 && nk == sg::NARROW_NONE && !k_split && work_floats >= sg::presplit_floats(N, K) &&
      (reinterpret_cast<uintptr_t>(work) & 15) == 0) {
    sg::PresplitJobs jobs{};
    jobs.n = 1;
    jobs.job[0] = sg::PresplitJob{B, b_n, b_k, N, K, sg::presplit_npad(N), work};
    if (sg::launch_mlp_presplit(jobs, g.split_tf32, s) != cudaSuccess) return SG_ERR_CUDA;
    g.b_pre = work;
    g.b_npad = sg::presplit_npad(N);
    return sg::launch_mlp_gemm(g, s) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
  }
  return sg::launch_mlp_gemm_split(g, work, work_floats, s) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}
