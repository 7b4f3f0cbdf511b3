// Shared pieces of the reduced-precision NNS (tcgen05, sm_103a): operand
// packing, instruction and shared-memory descriptors, tensor-memory access,
// the per-consumer top-K and the certificate of the exact re-rank.
//
// Operand layout ("K-major, no swizzle"): a tile of R rows and KB bytes per
// row is stored as KB/16 column blocks of R rows x 16 bytes; block c holds
// bytes [16c, 16c+16) of every row, rows 16 bytes apart.  Each 8-row x 16-byte
// piece is one core matrix; neighbouring core matrices are 128 bytes apart
// along M/N (stride byte offset) and R*16 bytes apart along K (leading byte
// offset).  A packed tile is one contiguous block, so a 1-D bulk copy (TMA)
// lands it in shared memory ready for the MMA descriptors.
#pragma once

#include <math_constants.h>

#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace nnsemd {

constexpr int TC_BM = 128;  // consumers per accumulator (MMA M)
constexpr int TC_K = 16;    // candidates kept per consumer

// FMT_BF16X3: every coordinate v as a high part h = bf16(v) and a low part
// l = bf16(v - h) (v - h is exact in FP32); a packed row holds 3d BF16
// values, [h(y), h(y), l(y)] for a consumer and [h(x), l(x), h(x)] for a
// supplier, so one BF16 contraction of length 3d gives
// <h(x), h(y)> + <l(x), h(y)> + <h(x), l(y)>, which differs from <x, y> by at
// most u^2 (3 + 2u + 2u^2) sum |x_k y_k| (u = 2^-8), against (2u + u^2) for
// a single BF16 copy.
enum TcFmt : int { FMT_F16 = 0, FMT_BF16 = 1, FMT_E4M3 = 2, FMT_BF16X3 = 3 };

__host__ __device__ inline int fmt_of_precision(int precision) {
  return precision == 1 ? FMT_BF16 : (precision == 2 ? FMT_F16 : (precision == 4 ? FMT_BF16X3 : FMT_E4M3));
}

// BF16 operands (kind::f16 with the BF16 type) and no per-row scale
__host__ __device__ constexpr bool fmt_is_bf16(int fmt) { return fmt == FMT_BF16 || fmt == FMT_BF16X3; }

// Values per coordinate in a packed row.
__host__ __device__ constexpr int fmt_parts(int fmt) { return fmt == FMT_BF16X3 ? 3 : 1; }

NNS_DEV uint16_t to_bits16(float v, int fmt) {
  if (fmt_is_bf16(fmt)) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  return __half_as_ushort(__float2half_rn(v));
}

NNS_DEV uint8_t to_e4m3(float v) { return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3); }

// Per-row scale (a power of two) for FP16 / FP8: the largest |v| of the row
// maps into [2^7, 2^8).  BF16 has FP32's exponent range and uses 1.
NNS_DEV float row_scale(const float* row, int d, int fmt) {
  if (!row || fmt_is_bf16(fmt)) return 1.f;
  float mx = 0.f;
  for (int k = 0; k < d; ++k) mx = fmaxf(mx, fabsf(row[k]));
  if (!(mx > 0.f)) return 1.f;
  int e;
  frexpf(mx, &e);  // mx in [2^(e-1), 2^e)
  return ldexpf(1.f, e - 8);
}

// Value k (0 <= k < 3d) of a BF16X3 packed row: segment k / d of [h, h, l]
// (consumer, supplier = false) or [h, l, h] (supplier).
NNS_DEV float bf16x3_part(const float* row, int d, int k, bool supplier) {
  const int seg = k / d;
  const float v = row[k - seg * d];
  const float h = __bfloat162float(__float2bfloat16_rn(v));
  const bool low = supplier ? seg == 1 : seg == 2;
  return low ? v - h : h;
}

// Pack 16 bytes (block c) of one row into out (row r of tile t).  row == null
// writes zeros (padding).  `supplier` picks the BF16X3 segment order.
NNS_DEV void pack_block(const float* row, int d, int c, float s, int fmt, uint8_t* tile_base, int tile_rows, int r,
                        bool supplier = false) {
  alignas(16) uint8_t bytes[16];
  if (fmt == FMT_BF16X3) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = c * 8 + e;
      const uint16_t b = to_bits16((row && k < 3 * d) ? bf16x3_part(row, d, k, supplier) : 0.f, fmt);
      bytes[2 * e] = (uint8_t)(b & 0xff);
      bytes[2 * e + 1] = (uint8_t)(b >> 8);
    }
  } else if (fmt == FMT_E4M3) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = c * 16 + e;
      bytes[e] = to_e4m3((row && k < d) ? row[k] / s : 0.f);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = c * 8 + e;
      const uint16_t b = to_bits16((row && k < d) ? row[k] / s : 0.f, fmt);
      bytes[2 * e] = (uint8_t)(b & 0xff);
      bytes[2 * e + 1] = (uint8_t)(b >> 8);
    }
  }
  *reinterpret_cast<uint4*>(tile_base + (size_t)c * tile_rows * 16 + (size_t)r * 16) =
      *reinterpret_cast<const uint4*>(bytes);
}

// FP32 squared norm (sequential fma) and L1 norm of a row.
NNS_DEV void row_norms(const float* row, int d, float& l2sq, float& l1) {
  float acc = 0.f, a1 = 0.f;
  for (int k = 0; k < d; ++k) {
    acc = __fmaf_rn(row[k], row[k], acc);
    a1 = __fadd_rn(a1, fabsf(row[k]));
  }
  l2sq = acc;
  l1 = a1;
}

// --------------------------------------------------------------------------
// tcgen05 helpers
// --------------------------------------------------------------------------

NNS_DEV uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  // base offset 0, relative LBO, swizzle mode 0 (none)
  return d;
}

// Instruction descriptor: D = F32, A and B of type `ab` (kind::f16: 0 = F16,
// 1 = BF16; kind::f8f6f4: 0 = E4M3), both K-major, N = n, M = m.
NNS_DEV uint32_t make_idesc(int ab, int m, int n) {
  return (1u << 4) | ((uint32_t)ab << 7) | ((uint32_t)ab << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

template <int FMT>
NNS_DEV void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  if (FMT == FMT_E4M3) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

NNS_DEV void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Wait for a phase, suspended in the barrier between polls: each try_wait
// carries a time hint of hint_ns, so the thread sleeps until the phase
// completes (and wakes at once then) or the hint runs out.  Gives up after
// `limit` polls (about a second with the default hint).
NNS_DEV bool mbar_wait_sleep(uint64_t* bar, unsigned parity, unsigned hint_ns = 1000u, unsigned limit = 1u << 20) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    if (ok) return true;
  }
  return false;
}

NNS_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

NNS_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
NNS_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

NNS_DEV void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

NNS_DEV void tmem_dealloc(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

NNS_DEV void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The same load without its wait: several loads go out back to back, then
// one tmem_ld_wait.  The registers must not be read before that wait, so the
// wait takes every destination block as an in/out operand of an (empty)
// ordered asm, which keeps the compiler from moving a read above it.
NNS_DEV void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

NNS_DEV void tmem_regs_after_wait(uint32_t (&r)[16]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
}

template <int NB>
NNS_DEV void tmem_ld_wait(uint32_t (&r)[NB][16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int b = 0; b < NB; ++b) tmem_regs_after_wait(r[b]);
}

// Make this thread's generic-proxy global writes visible to later bulk
// copies (async proxy) issued after a barrier.
NNS_DEV void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Unsigned image of a float that orders like the float itself (negative
// values included): flip every bit of a negative value, the sign bit of a
// non-negative one.
NNS_DEV unsigned ordered_bits(float v) {
  const unsigned b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Insert (v, p) into an ascending top-K list kept in registers; equal values
// keep their arrival order.
template <int K>
NNS_DEV void topk_insert(float (&tv)[K], int (&tp)[K], float v, int p) {
  if (!(v < tv[K - 1])) return;
  float nv = v;
  int np = p;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (nv < tv[k]) {
      const float fv = tv[k];
      const int fp = tp[k];
      tv[k] = nv;
      tp[k] = np;
      nv = fv;
      np = fp;
    }
  }
}

// Tagged top-K lists (the K2 epilogue).  A list entry is its approximate
// value with the low TAG bits of the FP32 pattern replaced by a tag; the tag
// names a slot of a per-thread table that holds the supplier position.  Tags
// of the entries in the list are distinct, so entries never compare equal
// and the list is kept by minima and maxima alone (no positions to move).
// The tag moves a value by less than 2^TAG units in the last place; every
// bound read from a list goes through tag_floor, the smallest value that
// shares the entry's other bits, which is at most the entry's exact value.
template <int KL>
struct TagList {
  static constexpr int TAG = KL <= 8 ? 4 : 5;  // 2^TAG >= KL + 1 tags
  static constexpr int NTAG = 1 << TAG;
  static constexpr unsigned MASK = NTAG - 1;
};

// FP32 bit patterns on either side (the host build serves the CPU tests)
__host__ __device__ inline unsigned f32_bits(float v) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(v);
#else
  unsigned u;
  memcpy(&u, &v, sizeof u);
  return u;
#endif
}

__host__ __device__ inline float f32_of_bits(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float v;
  memcpy(&v, &u, sizeof v);
  return v;
#endif
}

__host__ __device__ inline float tag_floor(float v, unsigned mask) {
  const unsigned u = f32_bits(v);
  return f32_of_bits((u & 0x80000000u) ? (u | mask) : (u & ~mask));
}

// Insert value v (finite) of supplier position pos: a free tag takes the
// position, the tagged value c enters the ascending list, and the entry
// pushed out (+inf while the list is not full, or c itself when it is above
// every entry) frees its tag.  All comparisons with c are taken first (the
// list is ascending and its entries distinct, so they read false ... false,
// true ... true), then every slot picks its new entry at once: a shallow
// chain instead of one comparison after another.  `table` points at this
// thread's tag 0 slot; slots are `stride` apart.
template <int KL>
__host__ __device__ inline void tag_insert(float (&tv)[KL], unsigned& used, int* table, int stride, float v,
                                           int pos) {
  using T = TagList<KL>;
#ifdef __CUDA_ARCH__
  const unsigned t = (unsigned)__ffs(~used) - 1u;
#else
  const unsigned t = (unsigned)__builtin_ffs((int)~used) - 1u;
#endif
  used |= 1u << t;
  table[t * stride] = pos;
  const float c = f32_of_bits((f32_bits(v) & ~T::MASK) | t);
  bool before[KL];
#pragma unroll
  for (int k = 0; k < KL; ++k) before[k] = c < tv[k];
  const float out = before[KL - 1] ? tv[KL - 1] : c;
#pragma unroll
  for (int k = KL - 1; k > 0; --k) tv[k] = before[k] ? (before[k - 1] ? tv[k - 1] : c) : tv[k];
  tv[0] = before[0] ? c : tv[0];
  if (!(out > 3.402823466e38f)) used &= ~(1u << (f32_bits(out) & T::MASK));
}

// --------------------------------------------------------------------------
// the certificate
//
// The epilogue ranks suppliers by a lower bound of the approximate distance:
//   v'_ij = |x_i|^2 - 2 s_i s_j <x^_i, y^_j> - c_j |x_i|,
//   c_j   = 2 Q |y_j|,
// where the subtracted term bounds the quantisation error of the dot product
// for this very pair (|<x~,y~> - <x,y>| <= Q |x| |y|, Q = 2u + u^2 for one
// rounded copy per side, u^2 (3 + 2u + 2u^2) for the BF16X3 split, by
// Cauchy-Schwarz; it enters twice).  Every supplier outside the K candidates
// has v' >= tau (the K-th smallest).  Its true squared distance d2 (of the
// float inputs) is therefore >= ny + tau - E, with E bounding what remains:
//   gamma (ny + rx^2)                         FP32 norms (sequential fma)
//   2 (eta terms)                             absolute rounding floor of the
//                                             operand format (subnormals,
//                                             times the row scale)
//   2 K 2^-22 |x~| |y~|                       tensor-core accumulation
//                                             (K = d, 3d for BF16X3; |x~|,
//                                             |y~| the packed rows' norms)
//   2 u32 (rx^2 + 2 |x~||y~| + c rx)          the epilogue's FP32 roundings
// (u = the operand format's unit roundoff, u32 = 2^-24, rx = max |x_i|,
// rx1 = max |x_i|_1 over the active suppliers).  Its FP32 key is >= d2 (1 -
// gamma) (gamma bounds the relative rounding of the sequential FP32 key), so
// the best exact candidate key is certified when strictly below
// (ny + tau - E)(1 - gamma).
// --------------------------------------------------------------------------

// (host and device: the CPU tests evaluate the certificate's arithmetic too)
__host__ __device__ inline double quant_unit(int fmt) {
  return fmt_is_bf16(fmt) ? 0x1p-8 : (fmt == FMT_F16 ? 0x1p-11 : 0x1p-4);
}

// Q with |<x~, y~> - <x, y>| <= Q sum |x_k y_k| <= Q |x| |y| for the dot
// product the format computes: 2u + u^2 for one rounded copy of each side,
// u^2 (3 + 2u + 2u^2) for the BF16X3 split (see FMT_BF16X3).
__host__ __device__ inline double quant_err(int fmt) {
  const double u = quant_unit(fmt);
  return fmt == FMT_BF16X3 ? u * u * (3.0 + 2.0 * u + 2.0 * u * u) : 2.0 * u + u * u;
}

// Bound on |a| / |v| for a packed operand row a of a row v (rounding
// only): 1 + u for one copy; the BF16X3 row [h, h, l] or [h, l, h] has
// |a|^2 <= 2 (1 + u)^2 |v|^2 + (u + u^2)^2 |v|^2.
__host__ __device__ inline double quant_norm_factor(int fmt) {
  const double u = quant_unit(fmt);
  return fmt == FMT_BF16X3 ? 1.4142135623731 * (1.0 + u) + u + u * u : 1.0 + u;
}

// c_j of the epilogue, from the consumer's FP32 squared norm (rounded up).
NNS_DEV float quant_coeff(int fmt, float ny) {
  return (float)(2.0 * quant_err(fmt) * sqrt((double)ny) * (1.0 + 1e-4));
}

// |x| rounded up, from the FP32 squared norm (sequential fma, relative error
// below 2e-5 for d <= 300 and far below 1e-4 for any d the kernels serve).
NNS_DEV float norm_up(float l2sq) { return sqrtf(l2sq) * (1.f + 1e-4f); }

// gamma_d of the sequential FP32 key (relative rounding bound).
__host__ __device__ inline double certify_gamma(int d) {
  const double u32 = 0x1p-24;
  return d * u32 / (1.0 - d * u32);
}

// E of the certificate: everything but ny + tau, for one consumer against
// suppliers with the given maxima (it does not depend on tau, so a solver
// whose maxima stay fixed can compute it once per consumer).
__host__ __device__ inline double certify_E(int fmt, int d, double ny, double yl2, double yl1, double sy, double rx,
                                            double rx1, double sxm) {
  const double u32 = 0x1p-24;
  const double uq = quant_unit(fmt);
  const double gam = certify_gamma(d);
  const double kdim = (double)d * fmt_parts(fmt);  // length of the contraction
  // absolute rounding floor of one packed value (subnormals; times the row
  // scale for FP16 / FP8); BF16X3 rounds twice per coordinate
  const double eta_unit =
      fmt == FMT_BF16 ? 0x1p-134 : (fmt == FMT_BF16X3 ? 0x1p-132 : (fmt == FMT_F16 ? 0x1p-25 : 0x1p-10));
  const double eta_x = eta_unit * (fmt_is_bf16(fmt) ? 1.0 : sxm);
  const double eta_y = eta_unit * (fmt_is_bf16(fmt) ? 1.0 : sy);
  const double dot_eta =
      fmt == FMT_BF16X3 ? 3.0 * (eta_x * (2.0 * yl1 + eta_y * d) + 2.0 * eta_y * rx1)
                        : eta_x * (yl1 + eta_y * d) + eta_y * rx1 + eta_x * uq * yl1 + eta_y * uq * rx1;
  const double nf = quant_norm_factor(fmt);
  const double xt = nf * rx + eta_x * sqrt(kdim), yt = nf * yl2 + eta_y * sqrt(kdim);
  const double dot_acc = kdim * 0x1p-22 * xt * yt;
  const double c = 2.0 * quant_err(fmt) * yl2 * (1.0 + 1e-5);
  return gam * (ny + rx * rx) + 2.0 * (dot_eta + dot_acc) + 2.0 * u32 * (rx * rx + 2.0 * xt * yt + c * rx) +
         1e-30;
}

// The bound a best exact FP32 key must stay strictly below to be certified:
// (ny + tau - E)(1 - gamma)(1 - 2^-30) when positive (the last factor covers
// the rounding of this double-precision evaluation), else the non-positive
// ny + tau - E itself, which no key (>= 0) is below.
__host__ __device__ inline double certify_floor_from_E(double ny, float tau, double E, double gam) {
  const double base = ny + (double)tau - E;  // <= 0: no key is certified (keys are >= 0)
  return base > 0.0 ? base * (1.0 - gam) * (1.0 - 0x1p-30) : base;
}

__host__ __device__ inline double certify_floor(int fmt, int d, double ny, double yl2, double yl1, double sy,
                                                double rx, double rx1, double sxm, float tau) {
  return certify_floor_from_E(ny, tau, certify_E(fmt, d, ny, yl2, yl1, sy, rx, rx1, sxm), certify_gamma(d));
}

__host__ __device__ inline bool certify(int fmt, int d, double ny, double yl2, double yl1, double sy, double rx,
                                        double rx1, double sxm, float tau, float best_key) {
  if (!(tau <= 3.402823466e38f)) return true;  // tau = +inf: every supplier of every chunk was a candidate
  return (double)best_key < certify_floor(fmt, d, ny, yl2, yl1, sy, rx, rx1, sxm, tau);
}

}  // namespace nnsemd
