// Shared device definitions: complex type, launch constants, axis plans, device scalars.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hom {

// Programmatic dependent launch: the pass kernels are launched (launch_pass, ops.h) so that
// their CTAs may be scheduled while the kernel before them on the stream drains; each calls
// this before its first access to global memory and waits there until that kernel has
// completed and its writes are visible. For a kernel launched without that dependency the
// wait returns at once.
__device__ __forceinline__ void wait_prior_grid() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// complex value; aligned to its size so that loads and stores are single vector accesses
template <typename T>
struct __align__(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

constexpr int kThreads = 256;     // threads per CTA of every pass kernel
constexpr int kMaxStages = 16;    // radix stages per axis
constexpr int kMaxRadix = 31;     // largest supported prime factor of an axis length
constexpr int kMaxAxis = 1023;    // longest supported axis (shared-memory tiles)

// Division of 32-bit unsigned numerators by a fixed divisor d >= 1 with a multiply-high and two
// shifts (Granlund-Montgomery round-up method): l = ceil(log2 d), m = floor(2^32 (2^l - d)/d) + 1,
// q = (t + ((x - t) >> min(l, 1))) >> max(l - 1, 0) with t = mulhi(m, x); exact for all x.
struct FastDiv {
  unsigned mul;
  unsigned sh1, sh2;
};
inline __host__ __device__ FastDiv make_fastdiv(int d) {
  unsigned l = 0;
  while ((1u << l) < (unsigned)d) ++l;
  FastDiv f;
  f.mul = (unsigned)(((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1);
  f.sh1 = l > 0 ? 1u : 0u;
  f.sh2 = l > 0 ? l - 1 : 0u;
  return f;
}

// Radix plan of one axis of odd length n = prod radix[s]; pprev[s] = prod_{t<s} radix[t];
// fdm[s], fdp[s] divide by n / radix[s] and by pprev[s]; fdn, fdnh by n and (n + 1) / 2
// (all computed on the host).
struct AxisPlan {
  int n;
  int nst;
  int radix[kMaxStages];
  int pprev[kMaxStages];
  FastDiv fdm[kMaxStages];
  FastDiv fdp[kMaxStages];
  FastDiv fdn, fdnh;
};

inline __host__ void plan_fastdivs(AxisPlan* P) {
  for (int s = 0; s < P->nst; ++s) {
    P->fdm[s] = make_fastdiv(P->n / P->radix[s]);
    P->fdp[s] = make_fastdiv(P->pprev[s]);
  }
  P->fdn = make_fastdiv(P->n);
  P->fdnh = make_fastdiv((P->n + 1) / 2);
}

// divisors of the line-pass loops (lines per CTA and its half), computed on the host
struct LineDiv {
  FastDiv lb, half;
};

// Scalars of one solve, resident on the device so that a captured iteration replays without
// host round trips. Written by the reduction finishers, read by every kernel of a step.
// components of a field: d for the vector fields of conductivity, d (d + 1) / 2 for the
// symmetric strain fields of elasticity (Mandel storage)
constexpr int kMaxComp = 6;

struct Scalars {
  double E[kMaxComp]; // macroscopic field (one entry per component)
  double omega;       // Richardson / Eyre-Milton parameter
  double alpha, beta; // CG / Chebyshev coefficients of the current step
  double rr;          // (r, r) of the current residual
  double pAp;         // (C p, p)
  double nb;          // ||b||
  double nE;          // ||E||
  double tol;         // epsilon
  double cheb_c, cheb_d;
  double last_res;    // last residual norm seen
  double last_inc;    // last increment norm seen
  double energy;      // (A(E+x), E+x) of the last energy evaluation
  double flux[kMaxComp];  // <A(E+x)>
  int it;             // completed iterations
  int done;           // 1 once stopped (converged or iteration limit)
  int converged;
  int maxit;
  int fixed;          // 1: run exactly maxit iterations, no stopping test
  int stop;           // 1 residual, 2 increment
  int which;          // Richardson: which of the two x buffers holds x_m
  int result;         // Richardson: buffer holding the returned iterate
  double* hist;       // per-iteration stopping quantity (device, hist_cap entries) or null
  int hist_cap;
  int nhist;          // entries recorded (may exceed hist_cap; the excess is not stored)
  // inner solves in potential coordinates (pcg_pot.cuh): the step length of the iterate update
  // u += alpha_u p and the coefficient of the direction update p = z + beta_p p that the next
  // step applies first, and 1 for Algorithm 3's coefficients (Chebyshev) instead of
  // Algorithm 2's
  double alpha_u, beta_p;
  int pot_cheb;
};

// PRE_CG_DOT / POST_CG_FUSED: the CG step (both precisions) with the vector update fused into
// the operator passes. In exact arithmetic (p, G A p) = (p, A p) for p in the range
// of the orthogonal projection G (every CG direction is), so (p, C p) and alpha come from the
// pre-operator pass and the inverse pass can update x and r and form (r, r) itself.
enum PreOp { PRE_AFFINE = 0, PRE_LINEAR = 1, PRE_CG = 2, PRE_EM = 3, PRE_IDENT = 4, PRE_CG_DOT = 5 };
enum PostOp { POST_STORE = 0, POST_RICH = 1, POST_CG = 2, POST_CHEB = 3, POST_EM = 4, POST_ADD = 5,
              POST_CG_FUSED = 6 };
enum ProjMode { PROJ_GAMMA = 0, PROJ_EM = 1 };
enum MatKind { MAT_PHASE_ISO = 0, MAT_PHASE_TENSOR = 1, MAT_FIELD = 2 };

// Conjugate gradients in potential coordinates (pcg_pot.cuh): the step's vectors u (iterate),
// r (residual), p (direction), complex half spectra in the layout of one spectrum component,
// and the modes of its two axis-0 kernels
template <typename T>
struct PotVecs {
  cpx<T>* u;
  cpx<T>* r;
  cpx<T>* p;
};
enum PotInvMode { POT_STEP = 0 /* u += alpha_u p, p = z +- beta p, lines of s = i p */,
                  POT_FIELD = 1 /* lines of s = i (u + alpha_u p) (x = D u, no update) */ };
enum PotFwdMode { POT_UPDATE = 0 /* r -= alpha q, (r, z), the step's coefficients */,
                  POT_INIT = 1 /* r = q (the right-hand side D* r_field), u = p = 0 */ };

// Coefficient view used by the pre/post operators, in the working precision T.
template <typename T>
struct MatView {
  int kind;
  int nphase;            // entries of the phase table (0: not known to the kernel)
  const uint8_t* ph8;
  const uint16_t* ph16;
  const T* table;        // nphase * nc * nc (tensor) or nphase (isotropic)
  const T* field;        // one scalar per node
  const T* inv;          // tensor phases with more than 3 components: nphase * nc * nc entries
                         // of (A_p + omega I)^{-1} for the Eyre-Milton post-operator, or null
};

// Accumulator of a dot product in FP64 accuracy. FP64 kernels accumulate in double; FP32
// kernels keep an unevaluated sum hi + lo of two floats and add each product with the
// error-free transformations TwoProduct (p + e = a b via one FMA) and TwoSum (Ogita, Rump &
// Oishi's compensated dot product), so the FP64 pipe is not used per element.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace hom
