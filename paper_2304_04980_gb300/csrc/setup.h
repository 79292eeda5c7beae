// Host-visible declarations of the setup stage (per-node inverses, node
// blocks of the splittings, banded block-Cholesky factors of Phi_bar).
#pragma once

#include "common.cuh"

namespace lq2d {

enum SetupStatus { kSetupNonFinite = 1, kSetupNotPD = 2, kSetupPhiNotPD = 4 };

struct SetupBuffers {
  // problem data (library-owned device copies)
  double* Aself;
  double* Anb;
  double* Bm;
  double* Qm;
  double* QTm;
  double* Rm;
  double* x0;
  // derived
  double* Qi;
  double* QTi;
  double* Sb;
  double* RiBt;
  double* AQ;
  double* QAt;
  double* M13;
  double* Om;
  double* fac;
  // two-ended (twisted) solve of Phi_bar, when enabled: the factor of the
  // reversed pair-row order, the interface blocks and the inverted interface
  // Schur complement per (v, class); NULL otherwise
  double* fac_rev;
  double* iface;
  double* sinv;
};

// pair-rows from which the two-ended solve applies (top and bottom halves
// of at least one row each around the two interface rows)
constexpr int kTwistedMinK = 4;

void launch_setup(const SetupBuffers& sb, int K, int N, int n, int m, int V, long long fac_rec,
                  long long fac_vc, int* d_status, cudaStream_t s);

}  // namespace lq2d
