// ffa_kinds.h -- launch kinds of the running-median de-reddening and of the peak finder,
// numbered after the periodogram's kinds (KernelKind), and the total count used by the
// launch accounting.
#pragma once

#include "ffa_internal.h"

namespace ffa {
constexpr int kMedianBuild = kNumKinds;      // the wavelet-matrix passes (many launches)
constexpr int kMedianQuery = kNumKinds + 1;  // the window queries
constexpr int kPeaks = kNumKinds + 2;        // peak finding (all its launches)
constexpr int kAllKinds = kNumKinds + 3;
}  // namespace ffa
