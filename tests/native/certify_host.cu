// Host entry points over the reduced-precision certificate of the library
// (csrc/tc_common.cuh), so the CPU tests can check its arithmetic against an
// exact restatement.  Built by tests/test_certificate.py; not part of the
// library.
#include "tc_common.cuh"

extern "C" double certify_floor_host(int fmt, int d, double ny, double yl2, double yl1, double sy, double rx,
                                     double rx1, double sxm, float tau) {
  return nnsemd::certify_floor(fmt, d, ny, yl2, yl1, sy, rx, rx1, sxm, tau);
}

extern "C" int certify_host(int fmt, int d, double ny, double yl2, double yl1, double sy, double rx, double rx1,
                            double sxm, float tau, float best_key) {
  return nnsemd::certify(fmt, d, ny, yl2, yl1, sy, rx, rx1, sxm, tau, best_key) ? 1 : 0;
}

// The K2 epilogue's tagged list over one stream of values, in arrival
// order: each value that beats the current last entry is inserted
// (tag_insert); at the end the tags are turned into positions and the values
// floored (floor = 0 leaves them tagged, to show what the floor is for).
// out_v / out_p get kl entries (+inf / -1 where the stream was shorter).
using nnsemd::f32_bits;
using nnsemd::tag_floor;
using nnsemd::tag_insert;
using nnsemd::TagList;

template <int KL>
static void tag_list_t(const float* vals, int n, int floor, float* out_v, int* out_p) {
  float tv[KL];
  int table[TagList<KL>::NTAG];
  unsigned used = 0u;
  for (int k = 0; k < KL; ++k) tv[k] = nnsemd::f32_of_bits(0x7f800000u);  // +inf
  for (int i = 0; i < n; ++i)
    if (vals[i] < tv[KL - 1]) tag_insert<KL>(tv, used, table, 1, vals[i], i);
  for (int k = 0; k < KL; ++k) {
    const bool real = !(tv[k] > 3.402823466e38f);
    out_p[k] = real ? table[f32_bits(tv[k]) & TagList<KL>::MASK] : -1;
    out_v[k] = (real && floor) ? tag_floor(tv[k], TagList<KL>::MASK) : tv[k];
  }
}

extern "C" int tag_list_host(const float* vals, int n, int kl, int floor, float* out_v, int* out_p) {
  if (kl == 8) {
    tag_list_t<8>(vals, n, floor, out_v, out_p);
    return 0;
  }
  if (kl == 16) {
    tag_list_t<16>(vals, n, floor, out_v, out_p);
    return 0;
  }
  return -1;
}
