// Device-side building blocks shared by the NNS-EMD kernels (sm_103a).
//
//  * the FP32 decision distance and the FP64 cost distance, each with one
//    fixed operation order (intrinsics only, so nothing is re-associated or
//    contracted by the compiler);
//  * an exact accumulator for sums of non-negative doubles, used for the
//    normalisation totals (Sec. II-A) and for R = sum f * D_ij (Alg. 1), so
//    both are correctly rounded whatever the order of accumulation;
//  * thin wrappers over mbarrier and the 1-D TMA bulk copy, with bounded
//    waits that raise an error flag instead of hanging.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define NNS_DEV __device__ __forceinline__

namespace nnsemd {

enum Metric : int { METRIC_L2 = 0, METRIC_SQL2 = 1, METRIC_L1 = 2 };

// Error bits raised on the device and read by the host after a call.
enum ErrFlag : unsigned {
  EF_NONFINITE = 1u,
  EF_NEGATIVE = 2u,
  EF_TIMEOUT = 4u,
  EF_CAPACITY = 8u,
  EF_ITER = 16u,
  EF_INTERNAL = 32u,
  EF_ZERO_MASS = 64u,
};

// Per-solve state in device memory; the host reads it through a pinned copy.
struct DevState {
  int mt, nt;                    // active supplier / consumer counts (written by compaction)
  unsigned long long nnz;        // flows (plan entries, cost terms) written
  unsigned err;                  // ErrFlag bits
  int nseg;                      // non-empty supplier groups this round
  int nbig;                      // groups longer than a warp this round
  int nmed;                      // groups of 9..32 consumers this round
  unsigned seg_cursor;           // member slots handed out this round
  long long rounds;              // rounds run on the device (finisher)
  long long pair_evals;          // sum of m_t * n_t over device-run rounds
  double total_a, total_b;       // normalisation totals (correctly rounded)
  double cost;                   // R (correctly rounded)
  double leftover;               // residual mass after the solve
  unsigned long long certified;  // reduced precision: consumer searches settled by the certificate
  unsigned long long fallbacks;  // reduced precision: consumer searches redone in FP32
  unsigned long long near_ties;  // reduced precision: exact re-rank overturned the approximate first choice
  unsigned long long widened;    // learned proposal: certified by the second tier
  unsigned ticket;               // blocks of the current compaction count done (reset by its last block)
};

// --------------------------------------------------------------------------
// distances
// --------------------------------------------------------------------------

// FP32 decision key: squared Euclidean for L2 / SQL2, L1 sum for L1.
// t_k = x_k - y_k; acc = t_0 * t_0; acc = fma(t_k, t_k, acc) (k ascending).
template <int METRIC>
NNS_DEV float key32(const float* x, const float* y, int d) {
  if (METRIC == METRIC_L1) {
    float acc = fabsf(__fsub_rn(x[0], y[0]));
    for (int k = 1; k < d; ++k) acc = __fadd_rn(acc, fabsf(__fsub_rn(x[k], y[k])));
    return acc;
  }
  float t = __fsub_rn(x[0], y[0]);
  float acc = __fmul_rn(t, t);
  for (int k = 1; k < d; ++k) {
    float u = __fsub_rn(x[k], y[k]);
    acc = __fmaf_rn(u, u, acc);
  }
  return acc;
}

// The FP32 key of key32<SQL2> (t = x_k - y_k, acc = t_0 t_0, then
// acc = fma(t_k, t_k, acc) in ascending k), read four coordinates at a time:
// x a 16-byte aligned global row, y a 16-byte aligned row (global or
// shared memory), d % 4 == 0.
NNS_DEV float key32_sql2_v4(const float* __restrict__ x, const float* y, int d) {
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* y4 = reinterpret_cast<const float4*>(y);
  float4 a = __ldg(x4), b = y4[0];
  float t = __fsub_rn(a.x, b.x);
  float acc = __fmul_rn(t, t);
  t = __fsub_rn(a.y, b.y);
  acc = __fmaf_rn(t, t, acc);
  t = __fsub_rn(a.z, b.z);
  acc = __fmaf_rn(t, t, acc);
  t = __fsub_rn(a.w, b.w);
  acc = __fmaf_rn(t, t, acc);
  for (int i = 1; i < (d >> 2); ++i) {
    a = __ldg(x4 + i);
    b = y4[i];
    t = __fsub_rn(a.x, b.x);
    acc = __fmaf_rn(t, t, acc);
    t = __fsub_rn(a.y, b.y);
    acc = __fmaf_rn(t, t, acc);
    t = __fsub_rn(a.z, b.z);
    acc = __fmaf_rn(t, t, acc);
    t = __fsub_rn(a.w, b.w);
    acc = __fmaf_rn(t, t, acc);
  }
  return acc;
}

// FP64 ground distance D_ij of the cost: the same steps in double, sqrt for L2.
NNS_DEV double cost_dist64(const float* x, const float* y, int d, int metric) {
  double acc;
  if (metric == METRIC_L1) {
    acc = fabs(__dsub_rn((double)x[0], (double)y[0]));
    for (int k = 1; k < d; ++k) acc = __dadd_rn(acc, fabs(__dsub_rn((double)x[k], (double)y[k])));
    return acc;
  }
  double t = __dsub_rn((double)x[0], (double)y[0]);
  acc = __dmul_rn(t, t);
  for (int k = 1; k < d; ++k) {
    double u = __dsub_rn((double)x[k], (double)y[k]);
    acc = __fma_rn(u, u, acc);
  }
  return metric == METRIC_L2 ? __dsqrt_rn(acc) : acc;
}

// Greedy-order and argmin key: (float bits of the FP32 key) << 32 | index.
// Non-negative floats order like their bit patterns, so a 64-bit unsigned
// minimum picks the smallest distance and then the smallest index.
NNS_DEV unsigned long long pack_key(float k, unsigned idx) {
  return ((unsigned long long)__float_as_uint(k) << 32) | idx;
}

// Random-protocol key of consumer j (original index) in round t: the upper
// half of SplitMix64 (Steele, Lea and Flood 2014) output number c + 1 of the
// generator seeded with `seed`, c = (t << 32) | j.  The generator adds
// 0x9E3779B97F4A7C15 to its state per step and mixes the state into its
// output; output k is therefore mix(seed + k * 0x9E3779B97F4A7C15).
NNS_DEV unsigned rp_key32(unsigned long long seed, long long t, int j) {
  const unsigned long long c = ((unsigned long long)t << 32) | (unsigned)j;
  unsigned long long z = seed + (c + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (unsigned)(z >> 32);
}

// One step of the greedy protocol (Alg. 1): f = min(s, c); s -= f; c -= f.
// Residuals are finite and never negative (they start positive and every
// step leaves x - x = +0 or the difference of the larger and the smaller),
// so their order is the order of their bit patterns, and the side that gave
// f becomes exactly +0: one FP64 subtraction, bit-identical to the two of
// the plain statement.  Returns f.
NNS_DEV bool residual_positive(double v) { return __double_as_longlong(v) > 0; }

NNS_DEV double greedy_step(double& s, double& c) {
  const long long sb = __double_as_longlong(s), cb = __double_as_longlong(c);
  const bool take_s = sb < cb;  // s < c: f = s
  const double f = take_s ? s : c;
  const double d = __dsub_rn(take_s ? c : s, f);
  s = take_s ? 0.0 : d;
  c = take_s ? d : 0.0;
  return f;
}

// --------------------------------------------------------------------------
// exact sum of non-negative finite doubles
//
// A double v = M * 2^(E-1075) (M < 2^53) is M << (E-1) in units of 2^-1074.
// That integer is split into 32-bit digits and added into 64-bit limbs
// (limb L holds digit weight 2^(32L) * 2^-1074); 64-bit limbs absorb 2^32
// additions of 32-bit digits without overflow.  The final carry propagation
// and round-to-nearest-even run in one thread.
// --------------------------------------------------------------------------

constexpr int XS_LIMBS = 68;

NNS_DEV void xs_digits(double v, int& limb, unsigned long long& c0, unsigned long long& c1,
                       unsigned long long& c2) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  int e = (int)((bits >> 52) & 0x7ff);
  unsigned long long mant = bits & 0xfffffffffffffULL;
  if (e) mant |= 1ULL << 52; else e = 1;
  int b = e - 1;
  limb = b >> 5;
  int sh = b & 31;
  unsigned long long lo = mant << sh;
  unsigned long long hi = sh ? (mant >> (64 - sh)) : 0ULL;
  c0 = lo & 0xffffffffULL;
  c1 = lo >> 32;
  c2 = hi;
}

// Add v (>= 0, finite) into an accumulator (shared or global memory).
NNS_DEV void xs_add(unsigned long long* acc, double v) {
  if (!(v > 0.0)) return;
  int L;
  unsigned long long c0, c1, c2;
  xs_digits(v, L, c0, c1, c2);
  if (c0) atomicAdd(acc + L, c0);
  if (c1) atomicAdd(acc + L + 1, c1);
  if (c2) atomicAdd(acc + L + 2, c2);
}

// The same add for the 32 lanes of a warp at once: every lane calls it (a
// lane with nothing to add passes 0).  Lanes whose values start at the same
// limb sum their digits by shuffles first (at most 32 digits below 2^32
// each: no overflow), then one of them adds the sums, so values that share
// an exponent cost three atomics per warp, not per lane.
static __device__ __noinline__ void xs_add_warp(unsigned long long* acc, double v) {  // one copy per file, not inlined at every site
  int L = -1;
  unsigned long long c0 = 0, c1 = 0, c2 = 0;
  if (v > 0.0) xs_digits(v, L, c0, c1, c2);
  const int lane = threadIdx.x & 31;
  const unsigned grp = __match_any_sync(0xffffffffu, L);
  if (grp == 0xffffffffu) {  // one limb for the whole warp (the same for every lane)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c0 += __shfl_xor_sync(0xffffffffu, c0, o);
      c1 += __shfl_xor_sync(0xffffffffu, c1, o);
      c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    if (L >= 0 && lane == 0) {
      if (c0) atomicAdd(acc + L, c0);
      if (c1) atomicAdd(acc + L + 1, c1);
      if (c2) atomicAdd(acc + L + 2, c2);
    }
    return;
  }
  unsigned long long s0 = 0, s1 = 0, s2 = 0;
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    const unsigned long long a0 = __shfl_sync(0xffffffffu, c0, k);
    const unsigned long long a1 = __shfl_sync(0xffffffffu, c1, k);
    const unsigned long long a2 = __shfl_sync(0xffffffffu, c2, k);
    if ((grp >> k) & 1u) {
      s0 += a0;
      s1 += a1;
      s2 += a2;
    }
  }
  if (L >= 0 && lane == __ffs(grp) - 1) {
    if (s0) atomicAdd(acc + L, s0);
    if (s1) atomicAdd(acc + L + 1, s1);
    if (s2) atomicAdd(acc + L + 2, s2);
  }
}

NNS_DEV unsigned long long xs_limb(const unsigned long long* a, int L) {
  return (L >= 0 && L < XS_LIMBS) ? a[L] : 0ULL;
}

// 64 bits of the normalised accumulator starting at bit position pos.
NNS_DEV unsigned long long xs_bits64(const unsigned long long* a, int pos) {
  int L = pos >> 5, r = pos & 31;
  unsigned long long lo = xs_limb(a, L) | (xs_limb(a, L + 1) << 32);
  unsigned long long hi = xs_limb(a, L + 2) | (xs_limb(a, L + 3) << 32);
  return r ? ((lo >> r) | (hi << (64 - r))) : lo;
}

// Correctly rounded value of the accumulator (single thread; a is modified).
NNS_DEV double xs_round(unsigned long long* a) {
  unsigned long long carry = 0;
  for (int L = 0; L < XS_LIMBS; ++L) {
    unsigned long long v = a[L] + carry;
    a[L] = v & 0xffffffffULL;
    carry = v >> 32;
  }
  int top = -1;
  for (int L = XS_LIMBS - 1; L >= 0; --L)
    if (a[L]) { top = L * 32 + (63 - __clzll((long long)a[L])); break; }
  if (top < 0) return 0.0;
  if (top <= 52) return __longlong_as_double((long long)xs_bits64(a, 0));
  int shift = top - 52;
  unsigned long long mant = xs_bits64(a, shift) & ((1ULL << 53) - 1);
  int rpos = shift - 1;
  unsigned long long round = (xs_bits64(a, rpos) & 1ULL);
  bool sticky = false;
  int Lr = rpos >> 5;
  for (int L = 0; L < Lr && !sticky; ++L) sticky = a[L] != 0;
  if (!sticky && (rpos & 31)) sticky = (a[Lr] & ((1ULL << (rpos & 31)) - 1)) != 0;
  if (round && (sticky || (mant & 1ULL))) {
    ++mant;
    if (mant >> 53) { mant >>= 1; ++shift; }
  }
  int E = shift + 1;
  if (E >= 2047) return __longlong_as_double(0x7ff0000000000000LL);
  return __longlong_as_double((long long)(((unsigned long long)E << 52) | (mant & ((1ULL << 52) - 1))));
}

// --------------------------------------------------------------------------
// mbarrier + 1-D bulk copy (TMA) helpers
// --------------------------------------------------------------------------

NNS_DEV unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

NNS_DEV void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

NNS_DEV void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

NNS_DEV void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

NNS_DEV bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for a phase with an iteration limit; returns false if it gave up.
NNS_DEV bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit = 1u << 22) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The same for a thread that usually waits long (a pipeline role that is
// not the bottleneck): after a short spin it sleeps between polls so that
// it leaves the issue slots to the warps doing the work.  Gives up after
// `limit` polls (about a second).
NNS_DEV bool mbar_wait_backoff(uint64_t* bar, unsigned parity, unsigned limit = 1u << 22) {
  for (unsigned it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it >= 16) __nanosleep(128);
  }
  return false;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
NNS_DEV void tma_load_1d(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// --------------------------------------------------------------------------
// packed FP32x2 arithmetic (sm_100+): two IEEE single-precision operations
// per instruction, lane-wise identical to the scalar _rn intrinsics.
// --------------------------------------------------------------------------

NNS_DEV unsigned long long f2_pack(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
NNS_DEV float f2_lo(unsigned long long v) { return __uint_as_float((unsigned)(v & 0xffffffffULL)); }
NNS_DEV float f2_hi(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }

NNS_DEV unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
NNS_DEV unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
NNS_DEV unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
NNS_DEV float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

}  // namespace nnsemd
