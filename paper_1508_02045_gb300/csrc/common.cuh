// Shared device definitions: complex type, launch constants, axis plans, device scalars.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hom {

template <typename T>
struct cpx {
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

// Radix plan of one axis of odd length n = prod radix[s]; pprev[s] = prod_{t<s} radix[t].
struct AxisPlan {
  int n;
  int nst;
  int radix[kMaxStages];
  int pprev[kMaxStages];
};

// Scalars of one solve, resident on the device so that a captured iteration replays without
// host round trips. Written by the reduction finishers, read by every kernel of a step.
struct Scalars {
  double E[3];        // macroscopic field
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
  double flux[3];     // <A(E+x)>
  int it;             // completed iterations
  int done;           // 1 once stopped (converged or iteration limit)
  int converged;
  int maxit;
  int fixed;          // 1: run exactly maxit iterations, no stopping test
  int stop;           // 1 residual, 2 increment
  int which;          // Richardson: which of the two x buffers holds x_m
  int result;         // Richardson: buffer holding the returned iterate
};

enum PreOp { PRE_AFFINE = 0, PRE_LINEAR = 1, PRE_CG = 2, PRE_EM = 3, PRE_IDENT = 4 };
enum PostOp { POST_STORE = 0, POST_RICH = 1, POST_CG = 2, POST_CHEB = 3, POST_EM = 4, POST_ADD = 5 };
enum ProjMode { PROJ_GAMMA = 0, PROJ_EM = 1 };
enum MatKind { MAT_PHASE_ISO = 0, MAT_PHASE_TENSOR = 1, MAT_FIELD = 2 };

// Coefficient view used by the pre/post operators. Phase tables live in double on the device
// and are converted per use; scalar fields are stored in the working precision T.
template <typename T>
struct MatView {
  int kind;
  const uint8_t* ph8;
  const uint16_t* ph16;
  const double* table;   // nphase * d * d (tensor) or nphase (isotropic)
  const T* field;        // one scalar per node
};

}  // namespace hom
