// Host helpers on the dense outputs of the library (no device code).
//
// sbg_zero_overlap: the coefficients of bin combinations in which two bins
// coincide (b1 = b2 in a 3PCF; any two of b1, b2, b3 in a 4PCF) hold the
// self-overlap terms of the grid estimator.  The paper's application figure
// (Sec. 4) ignores bin overlap and shows those diagonals as zero; this sets
// them to zero in place, leaving every other entry untouched.
#include "sarabande_gb300.h"

namespace {
constexpr int kMaxOutBins = 20;
}

extern "C" sbg_status sbg_zero_overlap(double* zeta, long long nouter, int nbins, int order, int ncomp) {
  if (!zeta || nouter < 0 || nbins < 1 || nbins > kMaxOutBins || (order != 3 && order != 4) ||
      (ncomp != 1 && ncomp != 2))
    return SBG_ERR_INVALID_ARG;
  const long long inner = order == 3 ? (long long)nbins * nbins : (long long)nbins * nbins * nbins;
  for (long long o = 0; o < nouter; ++o) {
    double* z = zeta + o * inner * ncomp;
    for (int b1 = 0; b1 < nbins; ++b1)
      for (int b2 = 0; b2 < nbins; ++b2) {
        if (order == 3) {
          if (b1 == b2)
            for (int q = 0; q < ncomp; ++q) z[((long long)b1 * nbins + b2) * ncomp + q] = 0.0;
          continue;
        }
        for (int b3 = 0; b3 < nbins; ++b3)
          if (b1 == b2 || b2 == b3 || b1 == b3)
            for (int q = 0; q < ncomp; ++q) z[(((long long)b1 * nbins + b2) * nbins + b3) * ncomp + q] = 0.0;
      }
  }
  return SBG_OK;
}
