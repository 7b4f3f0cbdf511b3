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
