// Labelled device tensors used by the H-bar build (internal).
#pragma once
#include <string>
#include <vector>

#include "gfcc_internal.cuh"

namespace gfcc {

// Non-owning labelled view: one character label per axis, row-major.
struct TV {
  double* p;
  std::string l;
  std::vector<int> d;
};

struct Tensor {
  std::string labels;
  std::vector<int> dims;
  DBuf<double> buf;
  Tensor(std::string l, std::vector<int> d);
  long long size() const;
  double* p() const { return buf.p; }
  // the same memory under other axis labels (relabelling = transposition in contractions)
  TV as(const std::string& l) const;
};

// C = alpha * sum A B + beta * C over the labels missing from C (no batch labels).
void contract(double alpha, const TV& A, const TV& B, double beta, const TV& C, cudaStream_t s);
// dst = alpha * src + beta * dst, matching axes by label
void perm(const TV& src, double alpha, double beta, const TV& dst, cudaStream_t s);

}  // namespace gfcc
