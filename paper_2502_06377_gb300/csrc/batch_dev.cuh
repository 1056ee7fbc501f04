// Batched inversion on the device (batch_dev.cu), internal.
#pragma once
#include "plan.cuh"

namespace ibmi {

// One matrix of a group: device A (p x p, lda; its lower triangle is read)
// and the caller's H (p x p, ldh).
struct BatchMat {
  const double* A;
  int64_t lda;
  double* H;
  int64_t ldh;
  int64_t p;
};

// n matrices padded to order pb with the partition (K, h), run in lockstep.
class DevGroup {
 public:
  DevGroup();
  ~DevGroup();
  DevGroup(const DevGroup&) = delete;
  DevGroup& operator=(const DevGroup&) = delete;
  // device bytes a group needs per matrix (estimate, for sizing groups)
  static size_t bytes_per_matrix(int64_t pb, int K, int64_t h);
  ibmi_status create(int64_t pb, int K, int64_t h, int n);
  // Inverts nrun <= n matrices (mixed precision, the options of `o`, Newton-Schulz
  // hand-over at ||I - A H||_F <= theta).  res[b]: each matrix's result;
  // fallback[b] = 1 for a matrix the lockstep rules leave unfinished (a stall
  // that needs the spectral-radius test, a failed tail, the sweep cap): the
  // caller runs it again on the single-matrix path.  H_b is written for every
  // matrix with res[b].status == IBMI_OK.  Synchronous on `st`.
  ibmi_status run(const BatchMat* mats, int nrun, const ibmi_batch_opts& o, double theta, cudaStream_t st,
                  ibmi_result* res, int* fallback);
  int capacity() const;
  size_t bytes() const;   // device bytes the group holds
  int rounds() const;   // rounds of the last run
  struct Impl;

 private:
  Impl* d;
};

}  // namespace ibmi
