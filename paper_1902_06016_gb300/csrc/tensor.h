// Labelled device tensors used by the H-bar build (internal).
#pragma once
#include <memory>
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

// The uploaded ground-state inputs and the H-bar elements that the IP (1h + 2h1p) and EA
// (1p + 2p1h) spaces share: tau, F_me, F_mi, F_ae, W_mbej and Y_mbej = t_jn^fb <mn||ef>
// (hbar.cu; o, v are the physical occupied and virtual counts).
struct HbarCommon {
  int o, v;
  std::unique_ptr<Tensor> eps, v_oooo, v_ooov, v_oovv, v_ovov, v_ovvv, t1, t2, l1, l2;
  Tensor tau, Fme, Fmi, Fae, Y, Wmbej;
  HbarCommon(int o_, int v_);
};
std::unique_ptr<HbarCommon> build_common(const HostInputs& in, int o, int v, cudaStream_t s);

}  // namespace gfcc
