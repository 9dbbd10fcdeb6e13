// Exact-slice FP64 GEMM on the tensor cores (see ozaki.cuh).
#include "ozaki.cuh"
#include "tc_gemm.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <cstdlib>

namespace gfcc {
namespace {

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

// ---- integer slicing -----------------------------------------------------------------------------
// Every step below is integer arithmetic on the FP64 bit patterns (FP64 instructions run on a narrow
// pipe on this GPU). For non-negative doubles the bit patterns order like the values, so the row
// maximum of |x| is an integer maximum, and the row exponent e (max |x| < 2^e, as frexp) is read
// from its exponent field; a row whose maximum is zero or subnormal is treated as zero.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}
constexpr int ZERO_ROW = -100000;   // row exponent marker of a zero (or subnormal-only) row
__device__ __forceinline__ int row_exponent(unsigned long long maxbits) {
  const int ex = (int)(maxbits >> 52);
  return ex == 0 ? ZERO_ROW : ex - 1022;
}
// Balanced base-128 digits of x relative to 2^(e - 6):  x ~ 2^(e-6) sum_{i<ns} a_i 2^(-7i), |a_i| <= 64.
// V = round(|x| 2^(6 - e + 7(ns-1))) is formed exactly from the mantissa (|V| <= 2^(6 + 7(ns-1)) < 2^56);
// digit i is V / 2^(7(ns-1-i)) rounded half up, V keeps the remainder (|remainder| <= 2^(shift-1)), and
// the signs of all digits follow x (so -x gives exactly the negated digits). a[i] holds digit i. The slice
// count NS is a template argument (no predicated iterations, constant shifts).
template <int NS>
__device__ __forceinline__ void digits_t(double x, int e, int (&a)[NS]) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long V = 0;
  if (ex != 0 && e != ZERO_ROW) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int t = ex - 1075 + 6 - e + 7 * (NS - 1);
    if (t >= 0) V = m << t;
    else if (t > -62) V = (m + (1LL << (-t - 1))) >> (-t);
  }
  const bool neg = bits < 0;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int shift = 7 * (NS - 1 - i);
    const long long d = (i < NS - 1) ? ((V + (1LL << (shift - 1))) >> shift) : V;
    V -= d << shift;
    a[i] = neg ? -(int)d : (int)d;
  }
}
// digits of two adjacent elements of a row, written as one bf16 pair per slot (k even)
template <int NS>
__device__ __forceinline__ void slice_pair(double x0, double x1, int e, __nv_bfloat16* __restrict__ o, long long kp,
                                           int reversed, long long k) {
  int a0[NS], a1[NS];
  digits_t<NS>(x0, e, a0);
  digits_t<NS>(x1, e, a1);
#pragma unroll
  for (int i = 0; i < NS; ++i)
    *reinterpret_cast<__nv_bfloat162*>(o + (long long)(reversed ? NS - 1 - i : i) * kp + k) =
        __halves2bfloat162(__int2bfloat16_rn(a0[i]), __int2bfloat16_rn(a1[i]));
}

// Real rows (row-major, row stride ldx, K used columns): one block per row (grid-stride) for long
// rows; slices [r][slot][kp] with slot = i (or ns-1-i when reversed), zeros for K <= k < kp.
template <int NS>
__global__ void __launch_bounds__(256) slice_kernel(const double* __restrict__ X, long long ldx, long long rows,
                                                    long long K, long long kp, int reversed,
                                                    __nv_bfloat16* __restrict__ out, int* __restrict__ expo) {
  __shared__ unsigned long long red[8];
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const double* x = X + r * ldx;
    unsigned long long mx = 0;
    for (long long k = threadIdx.x; k < K; k += blockDim.x) mx = max(mx, abs_bits(x[k]));
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
    const int e = row_exponent(mx);
    __syncthreads();
    if (threadIdx.x == 0) expo[r] = e == ZERO_ROW ? 0 : e;
    __nv_bfloat16* o = out + r * (long long)NS * kp;
    for (long long k = 2LL * threadIdx.x; k < kp; k += 2LL * blockDim.x)
      slice_pair<NS>(k < K ? x[k] : 0.0, k + 1 < K ? x[k + 1] : 0.0, e, o, kp, reversed, k);
  }
}
// The same for short rows: one warp per row.
template <int NS>
__global__ void __launch_bounds__(256) slice_rows_warp_kernel(const double* __restrict__ X, long long ldx,
                                                              long long rows, long long K, long long kp, int reversed,
                                                              __nv_bfloat16* __restrict__ out, int* __restrict__ expo) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const double* x = X + r * ldx;
  unsigned long long mx = 0;
  for (long long k = lane; k < K; k += 32) mx = max(mx, abs_bits(x[k]));
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const int e = row_exponent(mx);
  if (lane == 0) expo[r] = e == ZERO_ROW ? 0 : e;
  __nv_bfloat16* o = out + r * (long long)NS * kp;
  for (long long k = 2LL * lane; k < kp; k += 64)
    slice_pair<NS>(k < K ? x[k] : 0.0, k + 1 < K ? x[k + 1] : 0.0, e, o, kp, reversed, k);
}

// The same for a few long rows (fewer rows than it takes to occupy the GPU with a block each): the
// row maxima over chunks of SL_CH elements (atomic integer maxima of the bit patterns; rowmax zeroed by
// the caller), then the digits chunk by chunk.
constexpr long long SL_CH = 8192;
__global__ void __launch_bounds__(256) rowmax_chunk_kernel(const double* __restrict__ X, long long ldx, long long K,
                                                           unsigned long long* __restrict__ rowmax) {
  __shared__ unsigned long long red[8];
  const long long r = blockIdx.y, k0 = blockIdx.x * SL_CH, k1 = min(K, k0 + SL_CH);
  const double* x = X + r * ldx;
  unsigned long long mx = 0;
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) mx = max(mx, abs_bits(x[k]));
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
    if (mx > 0) atomicMax(rowmax + r, mx);
  }
}
template <int NS>
__global__ void __launch_bounds__(256) slice_chunk_kernel(const double* __restrict__ X, long long ldx, long long K,
                                                          long long kp, int reversed,
                                                          const unsigned long long* __restrict__ rowmax,
                                                          __nv_bfloat16* __restrict__ out, int* __restrict__ expo) {
  const long long r = blockIdx.y, k0 = blockIdx.x * SL_CH, k1 = min(kp, k0 + SL_CH);   // SL_CH is even
  const double* x = X + r * ldx;
  const int e = row_exponent(rowmax[r]);
  if (blockIdx.x == 0 && threadIdx.x == 0) expo[r] = e == ZERO_ROW ? 0 : e;
  __nv_bfloat16* o = out + r * (long long)NS * kp;
  for (long long k = k0 + 2LL * threadIdx.x; k < k1; k += 2LL * blockDim.x)
    slice_pair<NS>(k < K ? x[k] : 0.0, k + 1 < K ? x[k + 1] : 0.0, e, o, kp, reversed, k);
}

// the slice count of a launch as a template argument (2..8 slices)
template <typename F>
void with_ns(int ns, F&& f) {
  switch (ns) {
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    default: f(std::integral_constant<int, 8>{}); break;
  }
}

// ---- complex operands of zgemm_oz, sliced straight from their strided storage ----------------------
// Operand element (r, k) = Z[r * s_r + k * s_k] (complex), conjugated when conj. Real rows written:
//   mode 0 (left operand):  row r      = (Re, Im) interleaved along k
//   mode 1 (right operand): row r      = (Re, -Im)    and row R + r = (Im, Re)
// so that sum over the 2K real columns of left row m times right row n (or R + n) gives the real
// (imaginary) part of the complex product. Tiles of 32 rows x 64 complex k go through shared memory
// so that both the strided reads and the row-contiguous slice writes are coalesced.
constexpr int ZT_R = 32, ZT_K = 64;

__device__ __forceinline__ void load_ztile(const cplx* __restrict__ Z, long long s_r, long long s_k, int conj,
                                           long long R, long long K, long long r0, long long k0,
                                           cplx (*tile)[ZT_K + 1]) {
  if (s_r == 1) {   // consecutive rows are adjacent: threads along r
    const int tr = threadIdx.x & 31;
    for (int tk = threadIdx.x >> 5; tk < ZT_K; tk += blockDim.x >> 5) {
      const long long r = r0 + tr, k = k0 + tk;
      cplx v = make_cuDoubleComplex(0.0, 0.0);
      if (r < R && k < K) v = Z[r + k * s_k];
      if (conj) v.y = -v.y;
      tile[tr][tk] = v;
    }
  } else {          // threads along k
    for (int i = threadIdx.x; i < ZT_R * ZT_K; i += blockDim.x) {
      const int tr = i / ZT_K, tk = i % ZT_K;
      const long long r = r0 + tr, k = k0 + tk;
      cplx v = make_cuDoubleComplex(0.0, 0.0);
      if (r < R && k < K) v = Z[r * s_r + k * s_k];
      if (conj) v.y = -v.y;
      tile[tr][tk] = v;
    }
  }
}

// rowmax[r] = max over k of the bit patterns of |Re|, |Im| (atomic; rowmax zeroed by the caller)
__global__ void __launch_bounds__(256) zrowmax_kernel(const cplx* __restrict__ Z, long long s_r, long long s_k,
                                                      long long R, long long K,
                                                      unsigned long long* __restrict__ rowmax) {
  __shared__ cplx tile[ZT_R][ZT_K + 1];
  const long long r0 = (long long)blockIdx.y * ZT_R, k0 = (long long)blockIdx.x * ZT_K;
  load_ztile(Z, s_r, s_k, 0, R, K, r0, k0, tile);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int tr = warp; tr < ZT_R; tr += blockDim.x >> 5) {
    unsigned long long mx = 0;
    for (int tk = lane; tk < ZT_K; tk += 32) mx = max(mx, max(abs_bits(tile[tr][tk].x), abs_bits(tile[tr][tk].y)));
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0 && r0 + tr < R && mx > 0) atomicMax(rowmax + r0 + tr, mx);
  }
}

// Slices of row r at (r ns + slot) kp (row-major), or with slot_major at (slot rows_total + r) kp, where
// rows_total = R (mode 0) or 2R (mode 1): then slots 0..j of all rows form one contiguous block of rows.
template <int NS>
__global__ void __launch_bounds__(256) zslice_kernel(const cplx* __restrict__ Z, long long s_r, long long s_k,
                                                     int conj, long long R, long long K, int mode,
                                                     const unsigned long long* __restrict__ rowmax, long long kp,
                                                     int reversed, __nv_bfloat16* __restrict__ out,
                                                     int* __restrict__ expo, int slot_major = 0) {
  constexpr int ns = NS;
  __shared__ cplx tile[ZT_R][ZT_K + 1];
  const long long r0 = (long long)blockIdx.y * ZT_R, k0 = (long long)blockIdx.x * ZT_K;
  load_ztile(Z, s_r, s_k, conj, R, K, r0, k0, tile);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int tr = warp; tr < ZT_R; tr += blockDim.x >> 5) {
    const long long r = r0 + tr;
    if (r >= R) break;
    const int e = row_exponent(rowmax[r]);
    if (k0 == 0 && lane == 0) {
      expo[r] = e == ZERO_ROW ? 0 : e;
      if (mode == 1) expo[R + r] = e == ZERO_ROW ? 0 : e;
    }
    const long long rows_total = mode == 1 ? 2 * R : R;
    // element offset of slot 0 of a row and the distance between its slots
    const long long b0 = slot_major ? r * kp : r * (long long)ns * kp;
    const long long b1 = slot_major ? (R + r) * kp : (R + r) * (long long)ns * kp;
    const long long sstep = slot_major ? rows_total * kp : kp;
    __nv_bfloat16* o0 = out + b0;
    __nv_bfloat16* o1 = out + b1;
    for (int tk = lane; tk < ZT_K; tk += 32) {
      const long long k = k0 + tk;
      if (2 * k >= kp) break;
      const cplx v = tile[tr][tk];
      int are[NS], aim[NS];
      digits_t<NS>(v.x, e, are);
      digits_t<NS>(v.y, e, aim);
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        {
          const long long off = (long long)(reversed ? ns - 1 - i : i) * sstep + 2 * k;
          if (mode == 0) {
            *reinterpret_cast<__nv_bfloat162*>(o0 + off) = __halves2bfloat162(__int2bfloat16_rn(are[i]),
                                                                               __int2bfloat16_rn(aim[i]));
          } else {
            *reinterpret_cast<__nv_bfloat162*>(o0 + off) = __halves2bfloat162(__int2bfloat16_rn(are[i]),
                                                                               __int2bfloat16_rn(-aim[i]));
            *reinterpret_cast<__nv_bfloat162*>(o1 + off) = __halves2bfloat162(__int2bfloat16_rn(aim[i]),
                                                                               __int2bfloat16_rn(are[i]));
          }
        }
      }
    }
  }
}

// Output of an exact-slice product: real, out[m ldo + n] = beta out + P[m][n]; or complex (the real
// columns n and N + n of P hold the real and imaginary parts), C(m, n) = alpha P(m, n) + beta C(m, n).
struct OzOut {
  bool complex_out = false;
  double* out = nullptr;
  long long ldo = 0;
  double beta = 0.0;
  cplx* C = nullptr;
  long long scm = 0, scn = 0;
  cplx alpha = {1.0, 0.0}, cbeta = {0.0, 0.0};
  // the common cases, so that the output pass spends no FP64 multiplications on them (set by set_kinds):
  // alpha_kind 1: alpha = 1, 2: alpha = -1, 0: general; beta_kind 0: beta = 0, 1: beta = 1, 2: general
  int alpha_kind = 1, beta_kind = 0;
  void set_kinds() {
    alpha_kind = (alpha.y == 0.0 && alpha.x == 1.0) ? 1 : (alpha.y == 0.0 && alpha.x == -1.0) ? 2 : 0;
    if (complex_out) beta_kind = (cbeta.x == 0.0 && cbeta.y == 0.0) ? 0 : (cbeta.x == 1.0 && cbeta.y == 0.0) ? 1 : 2;
    else beta_kind = beta == 0.0 ? 0 : beta == 1.0 ? 1 : 2;
  }
};

// x 2^k by one multiplication with an exact power of two when 2^k is a normal number (ldexp otherwise)
__device__ __forceinline__ double scale_pow2(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * __longlong_as_double((long long)(k + 1023) << 52);
  return ldexp(x, k);
}
// sum_d S_d 2^(7 (nd - 1 - d)) for nd <= 8 per-diagonal integer sums |S_d| < 2^40: the first (up to four)
// and the remaining diagonals are combined exactly in two 64-bit integers (each below 2^62) and joined by
// one fused multiply-add, instead of an FP64 conversion and multiply-add per diagonal (FP64 is the scarce
// pipe on this GPU: the output passes were bound by it). The caller scales by 2^(-7 (nd - 1)).
__device__ __forceinline__ double diag_combine(const long long* S, int nd) {
  const int H = nd < 4 ? nd : 4;
  long long hi = 0, lo = 0;
#pragma unroll
  for (int d = 0; d < OZ_SLICES_MAX; ++d) {
    if (d < H) hi += S[d] * (1LL << (7 * (H - 1 - d)));
    else if (d < nd) lo += S[d] * (1LL << (7 * (nd - 1 - d)));
  }
  return fma((double)hi, __longlong_as_double((long long)(7 * (nd - H) + 1023) << 52), (double)lo);
}
// complex output value: alpha (re + i im) + beta C
__device__ __forceinline__ cplx out_value(const OzOut& o, double re, double im, const cplx* p) {
  cplx r;
  if (o.alpha_kind == 1) r = make_cuDoubleComplex(re, im);
  else if (o.alpha_kind == 2) r = make_cuDoubleComplex(-re, -im);
  else r = cuCmul(o.alpha, make_cuDoubleComplex(re, im));
  if (o.beta_kind == 1) {
    const cplx q = *p;
    r.x += q.x;
    r.y += q.y;
  } else if (o.beta_kind == 2) {
    r = cuCadd(r, cuCmul(o.cbeta, *p));
  }
  return r;
}
// real output value: v + beta out
__device__ __forceinline__ double out_value_real(const OzOut& o, double v, const double* p) {
  return o.beta_kind == 0 ? v : o.beta_kind == 1 ? v + *p : o.beta * (*p) + v;
}

// sum over the zs int32 split sums p[z stride], exactly in 64-bit integers; WARP: the lanes share the
// splits and every lane returns the total (integer sums do not depend on the grouping)
template <bool WARP>
__device__ __forceinline__ long long split_sum(const int* __restrict__ p, int zs, long long stride, int lane) {
  long long sum = 0;
  if constexpr (WARP) {
    for (int z = lane; z < zs; z += 32) sum += p[(long long)z * stride];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  } else {
    (void)lane;
    long long s1 = 0, s2 = 0, s3 = 0;   // four independent loads in flight
    int z = 0;
    for (; z + 4 <= zs; z += 4) {
      sum += p[(long long)z * stride];
      s1 += p[(long long)(z + 1) * stride];
      s2 += p[(long long)(z + 2) * stride];
      s3 += p[(long long)(z + 3) * stride];
    }
    for (; z < zs; ++z) sum += p[(long long)z * stride];
    sum += s1 + s2 + s3;
  }
  return sum;
}

// One diagonal of a column chunk (Np real columns): its split sums, weighted by scale = 2^(-7d), are
// added to the FP64 accumulator acc[m][n'] (MODE 0; first: acc is set), or, on the last diagonal, added
// to acc, scaled by 2^(ea[m] + eb[n'] - 12) and written to a real (MODE 1) or complex (MODE 2) output.
// One thread per element, or (WARP) one warp for outputs too small to occupy the GPU that have many K
// splits. Only the last diagonal needs the (m, n) of an element; 32-bit division when it fits.
template <typename I>
__device__ __forceinline__ void divmod(long long t, long long N, long long& m, long long& n) {
  m = (long long)((I)t / (I)N);
  n = t - m * N;
}
template <bool WARP, int MODE, typename I>
__global__ void __launch_bounds__(256) oz_accumulate_kernel(const int* __restrict__ part, int zs, long long M,
                                                            long long Np, double scale, int first,
                                                            double* __restrict__ acc, const int* __restrict__ ea,
                                                            const int* __restrict__ eb, OzOut o) {
  const long long stride = M * Np;
  const long long total = MODE == 2 ? M * (Np / 2) : stride;
  const int lane = threadIdx.x & 31;
  const bool writer = !WARP || lane == 0;
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const long long start = WARP ? gid >> 5 : gid, step = WARP ? nthreads >> 5 : nthreads;
  for (long long t = start; t < total; t += step) {
    if constexpr (MODE == 0) {
      double a = scale * (double)split_sum<WARP>(part + t, zs, stride, lane);
      if (!first) a = acc[t] + a;
      if (writer) acc[t] = a;
    } else if constexpr (MODE == 1) {
      double a = scale * (double)split_sum<WARP>(part + t, zs, stride, lane);
      if (!first) a = acc[t] + a;
      long long m, n;
      divmod<I>(t, Np, m, n);
      const double v = scale_pow2(a, ea[m] + eb[n] - 12);
      if (writer) {
        double* p = o.out + m * o.ldo + n;
        *p = out_value_real(o, v, p);
      }
    } else {
      const long long N = Np / 2;
      long long m, n;
      divmod<I>(t, N, m, n);
      const long long tr = m * Np + n, ti = tr + N;
      double ar = scale * (double)split_sum<WARP>(part + tr, zs, stride, lane);
      double ai = scale * (double)split_sum<WARP>(part + ti, zs, stride, lane);
      if (!first) {
        ar = acc[tr] + ar;
        ai = acc[ti] + ai;
      }
      const double re = scale_pow2(ar, ea[m] + eb[n] - 12), im = scale_pow2(ai, ea[m] + eb[N + n] - 12);
      if (writer) {
        cplx* p = o.C + m * o.scm + n * o.scn;
        *p = out_value(o, re, im, p);
      }
    }
  }
}
// All diagonals at once (their split sums held side by side: diagonal d at slabs + off[d], zs[d]
// splits of stride M Np each), summed and written to the output in one pass (MODE 1 real, 2 complex).
struct OzDiags {
  long long off[OZ_SLICES_MAX];
  int zs[OZ_SLICES_MAX];
  double scale[OZ_SLICES_MAX];
  int nd;
};
// sum_d 2^(-7d) (split sums of diagonal d), times 2^(7 (nd - 1)) (see diag_combine)
template <bool WARP>
__device__ __forceinline__ double diag_total(const int* __restrict__ slabs, const OzDiags& dg, long long stride,
                                             long long t, int lane) {
  long long S[OZ_SLICES_MAX];
#pragma unroll
  for (int d = 0; d < OZ_SLICES_MAX; ++d)
    S[d] = d < dg.nd ? split_sum<WARP>(slabs + dg.off[d] + t, dg.zs[d], stride, lane) : 0;
  return diag_combine(S, dg.nd);
}
template <bool WARP, int MODE, typename I>
__global__ void __launch_bounds__(256) oz_output_kernel(const int* __restrict__ slabs, OzDiags dg, long long M,
                                                        long long Np, const int* __restrict__ ea,
                                                        const int* __restrict__ eb, OzOut o) {
  const long long stride = M * Np;
  const long long total = MODE == 2 ? M * (Np / 2) : stride;
  const int lane = threadIdx.x & 31;
  const bool writer = !WARP || lane == 0;
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const long long start = WARP ? gid >> 5 : gid, step = WARP ? nthreads >> 5 : nthreads;
  for (long long t = start; t < total; t += step) {
    if constexpr (MODE == 1) {
      long long m, n;
      divmod<I>(t, Np, m, n);
      const double v = scale_pow2(diag_total<WARP>(slabs, dg, stride, t, lane), ea[m] + eb[n] - 12 - 7 * (dg.nd - 1));
      if (writer) {
        double* p = o.out + m * o.ldo + n;
        *p = out_value_real(o, v, p);
      }
    } else {
      const long long N = Np / 2;
      long long m, n;
      divmod<I>(t, N, m, n);
      const long long tr = m * Np + n;
      const int sh = -12 - 7 * (dg.nd - 1);
      const double re = scale_pow2(diag_total<WARP>(slabs, dg, stride, tr, lane), ea[m] + eb[n] + sh);
      const double im = scale_pow2(diag_total<WARP>(slabs, dg, stride, tr + N, lane), ea[m] + eb[N + n] + sh);
      if (writer) {
        cplx* p = o.C + m * o.scm + n * o.scn;
        *p = out_value(o, re, im, p);
      }
    }
  }
}
// The common case of one split per diagonal (a short K): the NS loads of an element are issued
// together, so that each thread keeps NS (complex: 2 NS) independent loads in flight.
template <int NS, int MODE, typename I>
__global__ void __launch_bounds__(256) oz_output1_kernel(const int* __restrict__ slabs, OzDiags dg, long long M,
                                                         long long Np, const int* __restrict__ ea,
                                                         const int* __restrict__ eb, OzOut o) {
  const long long stride = M * Np;
  const long long total = MODE == 2 ? M * (Np / 2) : stride;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    if constexpr (MODE == 1) {
      long long v[OZ_SLICES_MAX] = {};
#pragma unroll
      for (int d = 0; d < NS; ++d) v[d] = slabs[dg.off[d] + t];
      long long m, n;
      divmod<I>(t, Np, m, n);
      const double r = scale_pow2(diag_combine(v, NS), ea[m] + eb[n] - 12 - 7 * (NS - 1));
      double* p = o.out + m * o.ldo + n;
      *p = out_value_real(o, r, p);
    } else {
      const long long N = Np / 2;
      long long m, n;
      divmod<I>(t, N, m, n);
      const long long tr = m * Np + n, ti = tr + N;
      long long vr[OZ_SLICES_MAX] = {}, vi[OZ_SLICES_MAX] = {};
#pragma unroll
      for (int d = 0; d < NS; ++d) {
        vr[d] = slabs[dg.off[d] + tr];
        vi[d] = slabs[dg.off[d] + ti];
      }
      const int sh = -12 - 7 * (NS - 1);
      const double re = scale_pow2(diag_combine(vr, NS), ea[m] + eb[n] + sh);
      const double im = scale_pow2(diag_combine(vi, NS), ea[m] + eb[N + n] + sh);
      cplx* p = o.C + m * o.scm + n * o.scn;
      *p = out_value(o, re, im, p);
    }
  }
}
template <int MODE, typename I>
void launch_output1(int ns, int grid, cudaStream_t s, const int* slabs, const OzDiags& dg, long long M, long long Np,
                    const int* ea, const int* eb, const OzOut& o) {
  switch (ns) {
    case 2: oz_output1_kernel<2, MODE, I><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o); break;
    case 3: oz_output1_kernel<3, MODE, I><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o); break;
    case 4: oz_output1_kernel<4, MODE, I><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o); break;
    case 5: oz_output1_kernel<5, MODE, I><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o); break;
    case 6: oz_output1_kernel<6, MODE, I><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o); break;
    case 7: oz_output1_kernel<7, MODE, I><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o); break;
    default: oz_output1_kernel<8, MODE, I><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o); break;
  }
}

template <bool WARP, int MODE>
void launch_output(bool small, int grid, cudaStream_t s, const int* slabs, const OzDiags& dg, long long M,
                   long long Np, const int* ea, const int* eb, const OzOut& o) {
  if (small) oz_output_kernel<WARP, MODE, unsigned><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o);
  else oz_output_kernel<WARP, MODE, unsigned long long><<<grid, 256, 0, s>>>(slabs, dg, M, Np, ea, eb, o);
}

// ---- stacked form for a narrow right operand --------------------------------------------------------
// When B has few rows and A is large, one GEMM per A slice i multiplies it by B slices 0..ns-1-i
// stacked as rows (B sliced slot-major), so that A is read ns times instead of ns(ns+1)/2 times and the
// narrow B fills more of each tile. Partials of slice i: slabs + off[i], [zs[i]][M][ncol[i]] with
// ncol[i] = (ns - i) Np, B slice j in columns [j Np, (j + 1) Np). Diagonal d = i + j is summed exactly
// in 64-bit integers before the FP64 weighting, so the result equals the diagonal-by-diagonal one.
struct OzStack {
  long long off[OZ_SLICES_MAX];
  long long ncol[OZ_SLICES_MAX];
  int zs[OZ_SLICES_MAX];
  double scale[OZ_SLICES_MAX];
  int ns;
};
template <bool WARP>
__device__ __forceinline__ double stack_total(const int* __restrict__ slabs, const OzStack& st, long long M,
                                              long long Np, long long m, long long col, int lane) {
  long long S[OZ_SLICES_MAX];
#pragma unroll
  for (int d = 0; d < OZ_SLICES_MAX; ++d) {
    S[d] = 0;
    if (d < st.ns)
      for (int i = 0; i <= d; ++i)
        S[d] += split_sum<WARP>(slabs + st.off[i] + m * st.ncol[i] + (d - i) * Np + col, st.zs[i], M * st.ncol[i], lane);
  }
  return diag_combine(S, st.ns);   // times 2^(7 (ns - 1))
}
// complex output C(m, n) = alpha (re + i im) + beta C (real columns n and N + n of the Np = 2N)
template <bool WARP, typename I>
__global__ void __launch_bounds__(256) oz_stack_output_kernel(const int* __restrict__ slabs, OzStack st, long long M,
                                                              long long Np, const int* __restrict__ ea,
                                                              const int* __restrict__ eb, OzOut o) {
  const long long N = Np / 2, total = M * N;
  const int lane = threadIdx.x & 31;
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const long long start = WARP ? gid >> 5 : gid, step = WARP ? nthreads >> 5 : nthreads;
  for (long long t = start; t < total; t += step) {
    long long m, n;
    divmod<I>(t, N, m, n);
    const int sh = -12 - 7 * (st.ns - 1);
    const double re = scale_pow2(stack_total<WARP>(slabs, st, M, Np, m, n, lane), ea[m] + eb[n] + sh);
    const double im = scale_pow2(stack_total<WARP>(slabs, st, M, Np, m, N + n, lane), ea[m] + eb[N + n] + sh);
    if (!WARP || lane == 0) {
      cplx* p = o.C + m * o.scm + n * o.scn;
      *p = out_value(o, re, im, p);
    }
  }
}
// one split per slice product: all NS (NS + 1) / 2 loads of each part issued together
template <int NS, typename I>
__global__ void __launch_bounds__(256) oz_stack_output1_kernel(const int* __restrict__ slabs, OzStack st, long long M,
                                                               long long Np, const int* __restrict__ ea,
                                                               const int* __restrict__ eb, OzOut o) {
  constexpr int NQ = NS * (NS + 1) / 2;
  const long long N = Np / 2, total = M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long m, n;
    divmod<I>(t, N, m, n);
    int vr[NQ], vi[NQ];
#pragma unroll
    for (int d = 0, q = 0; d < NS; ++d)
#pragma unroll
      for (int i = 0; i <= d; ++i, ++q) {
        const int* p = slabs + st.off[i] + m * st.ncol[i] + (d - i) * Np + n;
        vr[q] = p[0];
        vi[q] = p[N];
      }
    long long sr[OZ_SLICES_MAX] = {}, si[OZ_SLICES_MAX] = {};
#pragma unroll
    for (int d = 0, q = 0; d < NS; ++d) {
#pragma unroll
      for (int i = 0; i <= d; ++i, ++q) {
        sr[d] += vr[q];
        si[d] += vi[q];
      }
    }
    const int sh = -12 - 7 * (NS - 1);
    const double re = scale_pow2(diag_combine(sr, NS), ea[m] + eb[n] + sh);
    const double im = scale_pow2(diag_combine(si, NS), ea[m] + eb[N + n] + sh);
    cplx* p = o.C + m * o.scm + n * o.scn;
    *p = out_value(o, re, im, p);
  }
}
template <typename I>
void launch_stack_output(int ns, bool one_split, bool warp, int grid, cudaStream_t s, const int* slabs,
                         const OzStack& st, long long M, long long Np, const int* ea, const int* eb, const OzOut& o) {
  if (one_split) {
    switch (ns) {
      case 5: oz_stack_output1_kernel<5, I><<<grid, 256, 0, s>>>(slabs, st, M, Np, ea, eb, o); return;
      case 6: oz_stack_output1_kernel<6, I><<<grid, 256, 0, s>>>(slabs, st, M, Np, ea, eb, o); return;
      case 7: oz_stack_output1_kernel<7, I><<<grid, 256, 0, s>>>(slabs, st, M, Np, ea, eb, o); return;
      default: break;
    }
  }
  if (warp) oz_stack_output_kernel<true, I><<<grid, 256, 0, s>>>(slabs, st, M, Np, ea, eb, o);
  else oz_stack_output_kernel<false, I><<<grid, 256, 0, s>>>(slabs, st, M, Np, ea, eb, o);
}

template <bool WARP, int MODE>
void launch_accumulate(bool small, int grid, cudaStream_t s, const int* part, int zs, long long M, long long Np,
                       double scale, int first, double* acc, const int* ea, const int* eb, const OzOut& o) {
  if (small)
    oz_accumulate_kernel<WARP, MODE, unsigned><<<grid, 256, 0, s>>>(part, zs, M, Np, scale, first, acc, ea, eb, o);
  else
    oz_accumulate_kernel<WARP, MODE, unsigned long long><<<grid, 256, 0, s>>>(part, zs, M, Np, scale, first, acc, ea,
                                                                             eb, o);
}

}  // namespace

namespace {
// algorithmic bytes of writing an M x Np output (a complex output holds Np / 2 complex columns), with a
// read of the old values when it is accumulated into
double out_bytes(const OzOut& o, long long M, long long Np) {
  if (o.complex_out) {
    const bool rd = o.cbeta.x != 0.0 || o.cbeta.y != 0.0;
    return (rd ? 2.0 : 1.0) * 16.0 * (double)M * (double)(Np / 2);
  }
  return (o.beta != 0.0 ? 2.0 : 1.0) * 8.0 * (double)M * (double)Np;
}

// Exact product of sliced rows into o. When the int32 split sums of all diagonals fit in 4 GB they are
// kept side by side and summed into the output in one pass. Otherwise the diagonal GEMMs run one at a
// time, each followed by its accumulation into an FP64 buffer, over column chunks that bound the
// split-sum memory (a complex output is one chunk, its real and imaginary columns being finalised
// together).
void oz_run(const SlicedRows& A, const SlicedRows& B, long long M, long long Np, const OzOut& o, OzWork& w,
            cudaStream_t s) {
  const int ns = A.ns;
  const double slab_bytes = oz_slab_bytes();
  const long long kp = A.kp, ld = (long long)ns * kp;
  const int max_splits = tc_exact_splits(M, Np, (long long)ns * kp);
  const __nv_bfloat16* As = reinterpret_cast<const __nv_bfloat16*>(A.slices.p);
  const __nv_bfloat16* Bs = reinterpret_cast<const __nv_bfloat16*>(B.slices.p);
  if (4.0 * ns * max_splits * (double)M * (double)Np <= slab_bytes) {
    // every diagonal's split sums side by side, then one pass that sums them into the output: the
    // output is touched once instead of once per diagonal
    w.islabs.alloc((size_t)ns * max_splits * M * Np + 4 * ns);
    if (w.err.n == 0) { w.err.alloc(1); w.err.zero(s); }
    OzDiags dg;
    dg.nd = ns;
    long long off = 0;
    for (int d = 0; d < ns; ++d) {
      const long long kd = (long long)(d + 1) * kp;
      const int zs = std::min(tc_exact_splits(M, Np, kd), max_splits);
      TcOperand a(As, M, kd, ld);
      TcOperand b(Bs + (long long)(ns - 1 - d) * kp, Np, kd, ld);
      dg.off[d] = off;
      dg.zs[d] = tc_gemm_exact(a, b, w.islabs.p + off, Np, M, Np, zs, M * Np, w.err.p, s, PROF_TC_SLICE);
      dg.scale[d] = ldexp(1.0, -7 * d);
      off = (off + (long long)zs * M * Np + 3) / 4 * 4;   // 16-byte aligned blocks (vector epilogue stores)
    }
    int splits = 0;
    for (int d = 0; d < ns; ++d) splits += dg.zs[d];
    const long long elements = o.complex_out ? M * (Np / 2) : M * Np;
    const bool warp = elements < 152LL * 256 && splits > 8 * ns;
    const int grid = warp ? (int)std::min<long long>(std::max<long long>((elements * 32 + 255) / 256, 1), 152LL * 32)
                          : grid_for(elements);
    const bool small = M * Np < (1LL << 32);
    // bytes: every int32 split sum read once, the output written once
    ProfScope pa(PROF_OZ_ACCUM, 4.0 * splits * (double)M * (double)Np + out_bytes(o, M, Np), s);
    if (splits == ns) {   // one split per diagonal
      if (o.complex_out) {
        if (small) launch_output1<2, unsigned>(ns, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
        else launch_output1<2, unsigned long long>(ns, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
      } else {
        if (small) launch_output1<1, unsigned>(ns, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
        else launch_output1<1, unsigned long long>(ns, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
      }
    } else if (o.complex_out) {
      if (warp) launch_output<true, 2>(small, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
      else launch_output<false, 2>(small, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
    } else {
      if (warp) launch_output<true, 1>(small, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
      else launch_output<false, 1>(small, grid, s, w.islabs.p, dg, M, Np, A.expo.p, B.expo.p, o);
    }
    GFCC_LAUNCH_CHECK();
    return;
  }
  // bytes of int32 split sums at a time (half the bound above)
  const long long slab_budget = (long long)std::max(1.0, std::min(2.0 * (1LL << 30), 0.5 * slab_bytes));
  long long nc = std::max<long long>(1, slab_budget / (4LL * M * max_splits));
  nc = std::min<long long>(Np, std::max<long long>(256, nc / 256 * 256));
  if (o.complex_out) nc = Np;
  w.islabs.alloc((size_t)max_splits * M * nc);
  w.acc.alloc((size_t)M * nc);
  if (w.err.n == 0) { w.err.alloc(1); w.err.zero(s); }
  for (long long n0 = 0; n0 < Np; n0 += nc) {
    const long long nn = std::min(nc, Np - n0);
    OzOut oc = o;
    if (!o.complex_out) oc.out = o.out + n0;
    for (int d = 0; d < ns; ++d) {
      // diagonal d: A slices 0..d against B slices d..0, concatenated along K
      const long long kd = (long long)(d + 1) * kp;
      const int zs = std::min(tc_exact_splits(M, nn, kd), max_splits);
      TcOperand a(As, M, kd, ld);
      TcOperand b(Bs + n0 * ld + (long long)(ns - 1 - d) * kp, nn, kd, ld);
      const int zeff = tc_gemm_exact(a, b, w.islabs.p, nn, M, nn, zs, M * nn, w.err.p, s, PROF_TC_SLICE);
      const double scale = ldexp(1.0, -7 * d);
      const int first = d == 0 ? 1 : 0;
      const int mode = d < ns - 1 ? 0 : (o.complex_out ? 2 : 1);
      const long long elements = mode == 2 ? M * (nn / 2) : M * nn;
      const bool warp = elements < 152LL * 256 && zeff > 8;
      const int grid = warp ? (int)std::min<long long>(std::max<long long>((elements * 32 + 255) / 256, 1), 152LL * 32)
                            : grid_for(elements);
      const bool small = M * nn < (1LL << 32);
      const int* eb = B.expo.p + n0;
      // bytes: the split sums read, the FP64 accumulator read (after the first diagonal) and written (or,
      // on the last diagonal, the output written)
      ProfScope pa(PROF_OZ_ACCUM, 4.0 * zeff * (double)M * (double)nn + (first ? 0.0 : 8.0 * (double)M * (double)nn) +
                                      (mode == 0 ? 8.0 * (double)M * (double)nn : out_bytes(oc, M, nn)), s);
      if (mode == 0) {
        if (warp) launch_accumulate<true, 0>(small, grid, s, w.islabs.p, zeff, M, nn, scale, first, w.acc.p, A.expo.p, eb, oc);
        else launch_accumulate<false, 0>(small, grid, s, w.islabs.p, zeff, M, nn, scale, first, w.acc.p, A.expo.p, eb, oc);
      } else if (mode == 1) {
        if (warp) launch_accumulate<true, 1>(small, grid, s, w.islabs.p, zeff, M, nn, scale, first, w.acc.p, A.expo.p, eb, oc);
        else launch_accumulate<false, 1>(small, grid, s, w.islabs.p, zeff, M, nn, scale, first, w.acc.p, A.expo.p, eb, oc);
      } else {
        if (warp) launch_accumulate<true, 2>(small, grid, s, w.islabs.p, zeff, M, nn, scale, first, w.acc.p, A.expo.p, eb, oc);
        else launch_accumulate<false, 2>(small, grid, s, w.islabs.p, zeff, M, nn, scale, first, w.acc.p, A.expo.p, eb, oc);
      }
      GFCC_LAUNCH_CHECK();
    }
  }
}

// Split counts of the stacked form (one GEMM per A slice against B slices 0..ns-1-i) and the bytes of
// their int32 partials.
void stack_splits(long long M, long long Np, long long kp, int ns, int (&zs)[OZ_SLICES_MAX], double& bytes) {
  bytes = 0.0;
  for (int i = 0; i < ns; ++i) {
    zs[i] = tc_exact_splits(M, (ns - i) * Np, kp);
    bytes += 4.0 * zs[i] * (double)M * (double)((ns - i) * Np) + 16.0;   // + alignment of each block
  }
}
// The stacked form pays when the A rows saved from re-reading, ns(ns-1)/2 kp bf16 per row, outweigh the
// extra partial sums it writes and reads back, about the same count times Np int32 per split, and its
// partials fit in 4 GB.
bool use_stacked(long long M, long long Np, long long kp, int ns) {
  int zs[OZ_SLICES_MAX];
  double bytes;
  stack_splits(M, Np, kp, ns, zs, bytes);
  return kp >= 4LL * Np * zs[0] && bytes <= oz_slab_bytes();
}
// Exact complex product in the stacked form: A sliced row-major (normal order), Bsm sliced slot-major
// (normal order) with Np = 2N rows per slot.
void oz_run_stacked(const SlicedRows& A, const SlicedRows& Bsm, long long M, long long Np, const OzOut& o,
                    OzWork& w, cudaStream_t s) {
  const int ns = A.ns;
  const long long kp = A.kp, ld = (long long)ns * kp;
  int zs[OZ_SLICES_MAX];
  double bytes;
  stack_splits(M, Np, kp, ns, zs, bytes);
  w.islabs.alloc((size_t)(bytes / 4.0));
  if (w.err.n == 0) { w.err.alloc(1); w.err.zero(s); }
  const __nv_bfloat16* As = reinterpret_cast<const __nv_bfloat16*>(A.slices.p);
  const __nv_bfloat16* Bs = reinterpret_cast<const __nv_bfloat16*>(Bsm.slices.p);
  OzStack st;
  st.ns = ns;
  long long off = 0;
  bool one_split = true;
  int splits = 0;
  for (int i = 0; i < ns; ++i) {
    const long long nc = (ns - i) * Np;
    TcOperand a(As + (long long)i * kp, M, kp, ld);
    TcOperand b(Bs, nc, kp, kp);
    st.off[i] = off;
    st.ncol[i] = nc;
    st.zs[i] = tc_gemm_exact(a, b, w.islabs.p + off, nc, M, nc, zs[i], M * nc, w.err.p, s, PROF_TC_SLICE);
    st.scale[i] = ldexp(1.0, -7 * i);
    // the GEMM epilogue stores rows of four int32 at once where ncol is a multiple of 4: every block
    // of partials starts on 16 bytes
    off = (off + (long long)zs[i] * M * nc + 3) / 4 * 4;
    one_split = one_split && st.zs[i] == 1;
    splits += st.zs[i];
  }
  const long long elements = M * (Np / 2);
  const bool warp = !one_split && elements < 152LL * 256 && splits > 8 * ns;
  const int grid = warp ? (int)std::min<long long>(std::max<long long>((elements * 32 + 255) / 256, 1), 152LL * 32)
                        : grid_for(elements);
  double part_bytes = 0.0;
  for (int i = 0; i < ns; ++i) part_bytes += 4.0 * st.zs[i] * (double)M * (double)st.ncol[i];
  ProfScope pa(PROF_OZ_ACCUM, part_bytes + out_bytes(o, M, Np), s);
  if (M * Np < (1LL << 32))
    launch_stack_output<unsigned>(ns, one_split, warp, grid, s, w.islabs.p, st, M, Np, A.expo.p, Bsm.expo.p, o);
  else
    launch_stack_output<unsigned long long>(ns, one_split, warp, grid, s, w.islabs.p, st, M, Np, A.expo.p,
                                            Bsm.expo.p, o);
  GFCC_LAUNCH_CHECK();
}
}  // namespace

double oz_slab_bytes() {
  double v = 4.0 * (1LL << 30);
  if (const char* env = getenv("GFCC_OZ_SLAB_BYTES")) v = atof(env);
  return v;
}

double oz_min_macs() {
  double v = 1e9;
  if (const char* env = getenv("GFCC_OZ_MIN_MACS")) v = atof(env);
  return v;
}

namespace {
struct ZSliceCache {   // slices of a left operand kept for several products with it
  SlicedRows sa;
  bool valid = false;
  const cplx* A = nullptr;   // the operand they were made from (checked on reuse)
  long long M = 0, K = 0, sam = 0, sak = 0;
  int ns = 0;
  bool conjA = false;
};
struct ZWork {          // buffers of zgemm_oz, kept between calls (grow-only)
  SlicedRows sa, sb;
  DBuf<unsigned long long> mxa, mxb;
  OzWork w;
  ZSliceCache cache[2];
};
}  // namespace

void* zgemm_work(gfcc_ctx* c) {
  if (!c->zwork) c->zwork = new ZWork();
  return c->zwork;
}
void* zgemm_slice_cache(gfcc_ctx* c, int i) {
  GFCC_CHECK(i == 0 || i == 1, GFCC_ERR_ARG, "zgemm_slice_cache: index");
  return &static_cast<ZWork*>(zgemm_work(c))->cache[i];
}
void zgemm_slice_cache_reset(void* cache) { static_cast<ZSliceCache*>(cache)->valid = false; }
void zgemm_work_free(gfcc_ctx* c) {
  delete static_cast<ZWork*>(c->zwork);
  c->zwork = nullptr;
}

void zgemm_oz(const ZGemmDesc& g, int ns, cudaStream_t s) {
  const long long M = g.M, N = g.N, K = g.K;
  GFCC_CHECK(g.batch == 1, GFCC_ERR_ARG, "zgemm_oz: no batches");
  GFCC_CHECK(ns >= 2 && ns <= OZ_SLICES_MAX, GFCC_ERR_ARG, "zgemm_oz: 2..8 slices");
  if (M <= 0 || N <= 0) return;
  ProfScope prof(PROF_OZ_ZGEMM, 8.0 * (double)M * (double)N * (double)K, s);
  ZWork local;
  ZWork& z = g.work ? *static_cast<ZWork*>(g.work) : local;
  ZSliceCache* cache = static_cast<ZSliceCache*>(g.a_cache);
  const bool reuse = cache && cache->valid && cache->A == g.A && cache->M == M && cache->K == K &&
                     cache->sam == g.sam && cache->sak == g.sak && cache->ns == ns && cache->conjA == g.conjA;
  SlicedRows& sa = cache ? cache->sa : z.sa;
  SlicedRows& sb = z.sb;
  sa.rows = M; sa.kp = tc_pad_k(TcKind::BF16, 2 * K); sa.ns = ns; sa.reversed = false;
  const bool stacked = use_stacked(M, 2 * N, sa.kp, ns);
  sb.rows = 2 * N; sb.kp = sa.kp; sb.ns = ns; sb.reversed = !stacked;
  if (!reuse) {
    sa.slices.alloc(sizeof(__nv_bfloat16) * M * ns * sa.kp);
    sa.expo.alloc(M);
  }
  sb.slices.alloc(sizeof(__nv_bfloat16) * 2 * N * ns * sb.kp);
  sb.expo.alloc(2 * N);
  {
    // bytes: each complex operand read once and its slices written once (A only when not cached)
    const double sb_bytes = 16.0 * (double)N * (double)K + 2.0 * (double)(2 * N) * ns * (double)sb.kp;
    const double sa_bytes = reuse ? 0.0 : 16.0 * (double)M * (double)K + 2.0 * (double)M * ns * (double)sa.kp;
    ProfScope ps(PROF_OZ_SLICE, sa_bytes + sb_bytes, s);
    DBuf<unsigned long long>& mxa = z.mxa;
    DBuf<unsigned long long>& mxb = z.mxb;
    mxa.alloc(M);
    mxb.alloc(N);
    GFCC_CUDA(cudaMemsetAsync(mxa.p, 0, sizeof(unsigned long long) * M, s));
    GFCC_CUDA(cudaMemsetAsync(mxb.p, 0, sizeof(unsigned long long) * N, s));
    const long long kt = (sa.kp / 2 + ZT_K - 1) / ZT_K;   // k tiles covering the padded width
    const long long kt_in = (K + ZT_K - 1) / ZT_K;
    GFCC_CHECK((M + ZT_R - 1) / ZT_R <= 65535 && (N + ZT_R - 1) / ZT_R <= 65535, GFCC_ERR_ARG, "zgemm_oz: too many rows");
    // A(m, k) = A[m sam + k sak]; B rows n: B(k, n) = B[k sbk + n sbn] -> r = n, s_r = sbn, s_k = sbk
    if (!reuse) {
      zrowmax_kernel<<<dim3((unsigned)kt_in, (unsigned)((M + ZT_R - 1) / ZT_R)), 256, 0, s>>>(g.A, g.sam, g.sak, M, K,
                                                                                           mxa.p);
      GFCC_LAUNCH_CHECK();
    }
    zrowmax_kernel<<<dim3((unsigned)kt_in, (unsigned)((N + ZT_R - 1) / ZT_R)), 256, 0, s>>>(g.B, g.sbn, g.sbk, N, K, mxb.p);
    GFCC_LAUNCH_CHECK();
    if (!reuse) {
      with_ns(ns, [&](auto NSc) {
        zslice_kernel<decltype(NSc)::value><<<dim3((unsigned)kt, (unsigned)((M + ZT_R - 1) / ZT_R)), 256, 0, s>>>(
            g.A, g.sam, g.sak, g.conjA ? 1 : 0, M, K, 0, mxa.p, sa.kp, 0,
            reinterpret_cast<__nv_bfloat16*>(sa.slices.p), sa.expo.p);
      });
      GFCC_LAUNCH_CHECK();
      if (cache) {
        cache->valid = true;
        cache->A = g.A; cache->M = M; cache->K = K; cache->sam = g.sam; cache->sak = g.sak;
        cache->ns = ns; cache->conjA = g.conjA;
      }
    }
    with_ns(ns, [&](auto NSc) {
      zslice_kernel<decltype(NSc)::value><<<dim3((unsigned)kt, (unsigned)((N + ZT_R - 1) / ZT_R)), 256, 0, s>>>(
          g.B, g.sbn, g.sbk, g.conjB ? 1 : 0, N, K, 1, mxb.p, sb.kp, stacked ? 0 : 1,
          reinterpret_cast<__nv_bfloat16*>(sb.slices.p), sb.expo.p, stacked ? 1 : 0);
    });
    GFCC_LAUNCH_CHECK();
  }
  OzOut o;
  o.complex_out = true;
  o.C = g.C;
  o.scm = g.scm;
  o.scn = g.scn;
  o.alpha = g.alpha;
  o.cbeta = g.beta;
  o.set_kinds();
  OzWork& w = z.w;
  if (stacked) oz_run_stacked(sa, sb, M, 2 * N, o, w, s);
  else oz_run(sa, sb, M, 2 * N, o, w, s);
  if (g.work) return;   // the caller checks the workspace's error flag (zgemm_work_check) later
  int herr = 0;
  GFCC_CUDA(cudaMemcpyAsync(&herr, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  GFCC_CHECK(herr == 0, GFCC_ERR_CUDA, "zgemm_oz: tensor-core pipeline wait timed out");
}

void zgemm_work_check(gfcc_ctx* c) {
  if (!c->zwork) return;
  ZWork* z = static_cast<ZWork*>(c->zwork);
  if (z->w.err.n == 0) return;
  int herr = 0;
  GFCC_CUDA(cudaMemcpyAsync(&herr, z->w.err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  GFCC_CHECK(herr == 0, GFCC_ERR_CUDA, "exact-slice GEMM: tensor-core pipeline wait timed out");
}

void oz_slice_into(const double* X, long long ldx, long long nrows, long long K, SlicedRows& out, long long row0,
                   cudaStream_t s) {
  GFCC_CHECK(row0 >= 0 && row0 + nrows <= out.rows && K <= out.kp, GFCC_ERR_ARG, "oz_slice_into: out of range");
  if (nrows == 0) return;
  // bytes: the FP64 rows read once, their slices written once
  ProfScope prof(PROF_OZ_SLICE, 8.0 * (double)nrows * (double)K + 2.0 * (double)nrows * out.ns * (double)out.kp, s);
  __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out.slices.p) + row0 * out.ns * out.kp;
  if (out.kp <= 2048) {   // short rows: a warp per row
    with_ns(out.ns, [&](auto NSc) {
      slice_rows_warp_kernel<decltype(NSc)::value><<<(unsigned)((nrows * 32 + 255) / 256), 256, 0, s>>>(
          X, ldx, nrows, K, out.kp, out.reversed ? 1 : 0, o, out.expo.p + row0);
    });
  } else if (nrows < 152LL * 4 && nrows <= 65535) {   // few long rows: split each row over blocks
    DBuf<unsigned long long> mx;
    mx.alloc(nrows);
    mx.zero(s);
    const long long chunks_in = (K + SL_CH - 1) / SL_CH, chunks = (out.kp + SL_CH - 1) / SL_CH;
    rowmax_chunk_kernel<<<dim3((unsigned)std::max<long long>(chunks_in, 1), (unsigned)nrows), 256, 0, s>>>(X, ldx, K,
                                                                                                         mx.p);
    GFCC_LAUNCH_CHECK();
    with_ns(out.ns, [&](auto NSc) {
      slice_chunk_kernel<decltype(NSc)::value><<<dim3((unsigned)chunks, (unsigned)nrows), 256, 0, s>>>(
          X, ldx, K, out.kp, out.reversed ? 1 : 0, mx.p, o, out.expo.p + row0);
    });
    GFCC_LAUNCH_CHECK();
    GFCC_CUDA(cudaStreamSynchronize(s));   // mx is released on return
    return;
  } else {
    const int grid = (int)std::min<long long>(nrows, 152LL * 16);
    with_ns(out.ns, [&](auto NSc) {
      slice_kernel<decltype(NSc)::value><<<grid, 256, 0, s>>>(X, ldx, nrows, K, out.kp, out.reversed ? 1 : 0, o,
                                                             out.expo.p + row0);
    });
  }
  GFCC_LAUNCH_CHECK();
}

void oz_slice(const double* X, long long ldx, long long rows, long long K, bool reversed, SlicedRows& out,
              cudaStream_t s, int ns) {
  GFCC_CHECK(ns >= 2 && ns <= OZ_SLICES_MAX, GFCC_ERR_ARG, "oz_slice: 2..8 slices");
  out.rows = rows;
  out.kp = tc_pad_k(TcKind::BF16, K);
  out.ns = ns;
  out.reversed = reversed;
  out.slices.alloc(sizeof(__nv_bfloat16) * std::max<long long>(rows, 1) * ns * out.kp);
  out.expo.alloc(std::max<long long>(rows, 1));
  oz_slice_into(X, ldx, rows, K, out, 0, s);
}

void oz_gemm(const SlicedRows& A, const SlicedRows& B, long long M, long long N, double* out, long long ldo,
             double beta, OzWork& w, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  GFCC_CHECK(!A.reversed && B.reversed && A.kp == B.kp && A.ns == B.ns, GFCC_ERR_ARG,
             "oz_gemm: operand slicing mismatch");
  GFCC_CHECK(A.rows >= M && B.rows >= N, GFCC_ERR_ARG, "oz_gemm: operand rows");
  OzOut o;
  o.out = out;
  o.ldo = ldo;
  o.beta = beta;
  o.set_kinds();
  oz_run(A, B, M, N, o, w, s);
}

}  // namespace gfcc
