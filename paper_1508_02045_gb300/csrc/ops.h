// Host-side launchers of the pass kernels, one instantiation per working precision
// (ops_f64.cu, ops_f32.cu). The host API (hom_api.cu) sequences them into operator
// applications and solver steps.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace hom {

struct OpArgs;
struct ProjGeom;
template <typename T> struct Fields;
template <typename T> struct ReqDesc;

// launch geometry of the kernels of one grid, chosen by the planner in hom_api.cu
struct PassGeom {
  int D;              // spatial dimension
  int NC;             // components of a field: D (vectors) or D (D + 1) / 2 (symmetric strains)
  int n[3];           // solve-grid order
  long long nodes;    // |grid|
  long long nlines;   // lines of the contiguous axis per component (|grid| / n[D-1])
  int nh;             // (n[D-1] + 1) / 2
  long long scs;      // spectrum component stride: nlines * nh
  int LB;             // lines per CTA in the line passes (even)
  int NTl;            // threads per CTA of the runtime-radix line passes (128 or 256)
  int TC1, TC1p, NT1;     // strided pass along axis 1 (D = 3): columns per CTA, padded pitch,
                          // threads per CTA
  int TCs0, TCs0p, NTs0;  // plain strided pass along axis 0 (prolongation, Ga assembly)
  int TC0, TC0p, NT0;     // projection pass (axis 0, all components)
  int TCq, TCqp, NTq;     // projection pass of the 3-D scalar problem (two lines a column)
};

template <typename T>
struct Ops {
  static cudaError_t upload_constants();
  static size_t smem_line(int n, int ncomp, int LB);
  static size_t smem_strided(int n, int TCp, int nst);
  static size_t smem_proj(int n, int D, int TCp, int nst);
  static size_t smem_proj_scalar(int n, int TCp);
  // launch geometry of every pass of a grid with axis plans `plan` for fields of nc components,
  // keeping each CTA's shared memory within `budget` bytes and its threads within `threads`
  // (<= kThreads); false if a pass cannot fit the device limit
  static bool plan_geometry(int D, const int* n, const AxisPlan* plan, size_t budget,
                            int threads, PassGeom* g, int nc = 0);
  static cudaError_t prepare(int maxD);  // raise dynamic shared memory limits

  // reqs / nreq: optional per-request descriptors of a batched launch (grid.z = nreq); the
  // direct arguments are then ignored where a descriptor provides them
  // partials: the per-CTA partials of (p, A p) written by PRE_CG_DOT (unused otherwise)
  static void line_fwd(const PassGeom& g, int pre, const Fields<T>& f, cpx<T>* S,
                       const AxisPlan& P, const cpx<T>* tw, int ncomp, const MatView<T>& mat,
                       Scalars* sc, const OpArgs& args, cudaStream_t st,
                       const ReqDesc<T>* reqs = nullptr, int nreq = 1,
                       double* partials = nullptr);
  // strided DFT along axis 1 (D = 3) or axis 0 (no projection) of ncomp components
  static void strided(const PassGeom& g, int axis, int inv, cpx<T>* S, const AxisPlan& P,
                      const cpx<T>* tw, int ncomp, const Scalars* sc, cudaStream_t st,
                      const ReqDesc<T>* reqs = nullptr, int nreq = 1);
  static void proj(const PassGeom& g, int mode, cpx<T>* S, const AxisPlan& P, const cpx<T>* tw,
                   const ProjGeom& pg, const Scalars* sc, cudaStream_t st,
                   const ReqDesc<T>* reqs = nullptr, int nreq = 1);
  // The 3-D scalar projection (PROJ_GAMMA) with two spectrum lines between the column passes
  // when both column axes have compile-time FP32 plans: axis-1 forward writes X_0 and
  // Y = k_1 X_1 + k_2 X_2, the projection reads and writes two lines, axis-1 inverse expands
  // them to three components. two_line_ok says whether the chain applies.
  static bool two_line_ok(const PassGeom& g, const AxisPlan& P0, const AxisPlan& P1);
  static void strided_two_line(const PassGeom& g, int inv, cpx<T>* S, const AxisPlan& P,
                               const cpx<T>* tw, const Scalars* sc, cudaStream_t st,
                               const ReqDesc<T>* reqs = nullptr, int nreq = 1);
  static void proj_two_line(const PassGeom& g, cpx<T>* S, const AxisPlan& P, const cpx<T>* tw,
                            const ProjGeom& pg, const Scalars* sc, cudaStream_t st,
                            const ReqDesc<T>* reqs = nullptr, int nreq = 1);
  static void line_inv(const PassGeom& g, int post, const cpx<T>* S, const Fields<T>& f,
                       const AxisPlan& P, const cpx<T>* tw, int ncomp, const MatView<T>& mat,
                       Scalars* sc, const OpArgs& args, double* partials, unsigned* counter,
                       int negate, cudaStream_t st, const ReqDesc<T>* reqs = nullptr,
                       int nreq = 1);
  // ncomp: components of x (the coefficient acts on ncomp-vectors)
  // alpha = (r, r) / (p, A p) from the nb per-CTA partials of (p, A p) (one CTA per request)
  static void cg_alpha(const double* partials, int nb, long long count, Scalars* sc,
                       cudaStream_t st, const ReqDesc<T>* reqs = nullptr, int nreq = 1);
  static void energy(int ncomp, const T* x, long long nodes, const MatView<T>& mat, Scalars* sc,
                     double* partials, unsigned* counter, int grid, cudaStream_t st);
  static void fill_const(T* x, long long nodes, int d, const Scalars* sc, cudaStream_t st);
  static void demote(const double* r64, T* r, T* p, T* x, long long len, long long nodes,
                     Scalars* sc, double* partials, unsigned* counter, int grid, cudaStream_t st);
  static void promote(double* x64, const T* dx, long long len, cudaStream_t st);
  static void convert_in(const double* src, T* dst, long long len, cudaStream_t st);
  static void convert_out(const T* src, double* dst, long long len, cudaStream_t st);
  static void crop_spectrum(const cpx<T>* Sm, cpx<T>* Sn, int D, int n0, int n1, int nh, int m0,
                            int m1, int mh, double scale, long long nlen, long long mlen,
                            cudaStream_t st);
  static void pad_spectrum(const cpx<T>* Sn, cpx<T>* Sm, int D, int n0, int n1, int nh, int m0,
                           int m1, int mh, double scale, long long nlen, long long mlen,
                           cudaStream_t st);
};

// FP32 kernels specialised at compile time for the two-stage plans of the usual axis lengths
// (ops_pair_f32.cu); the callers fall back to the runtime-radix kernels for everything else
bool pair_plan_f32(const AxisPlan& P);
cudaError_t pair_prepare_f32(int smem_cap);
// TMA waits that ran out on the current device since the last reset (tma.cuh)
unsigned tma_wait_errors(bool reset);
// on: announce 16 bytes more than each TMA tile copy delivers, so that its waits run out
void tma_debug_stall(bool on);
void pair_strided_f32(const AxisPlan& P, int inv, cpx<float>* S, const cpx<float>* tw,
                      long long C, long long es, long long bs, int batches, const Scalars* sc,
                      cudaStream_t st, const ReqDesc<float>* reqs, int nreq);
void pair_proj_f32(int D, int mode, bool two, const AxisPlan& P, cpx<float>* S,
                   const cpx<float>* tw, const ProjGeom& pg, const Scalars* sc, cudaStream_t st,
                   const ReqDesc<float>* reqs, int nreq);
// axis-1 pass of components 1 and 2 in the two-line chain of the 3-D scalar projection
void pair_strided2_f32(const AxisPlan& P, int inv, cpx<float>* S, const cpx<float>* tw,
                       long long C, long long es, long long bs, long long cs, int planes,
                       const Scalars* sc, cudaStream_t st, const ReqDesc<float>* reqs, int nreq);
// the line passes are specialised for D = 3 and the pre-/post-operators of the FP32 inner
// solves (CG, Chebyshev) and of plain operator applications
// D: components of the fields (3: vector fields of a 3-D grid; 6: strain fields of a 3-D
// grid, for the inner steps of the refinement)
inline bool pair_line_fwd_has(int D, int pre) {
  return (D == 3 && (pre == PRE_CG || pre == PRE_CG_DOT || pre == PRE_LINEAR)) ||
         (D == 6 && (pre == PRE_CG_DOT || pre == PRE_LINEAR));
}
inline bool pair_line_inv_has(int D, int post) {
  return (D == 3 && (post == POST_CG || post == POST_CG_FUSED || post == POST_CHEB ||
                     post == POST_STORE)) ||
         (D == 6 && (post == POST_CG_FUSED || post == POST_CHEB));
}
// returns the number of CTAs (the partials a PRE_CG_DOT pass writes)
int pair_line_fwd_f32(int D, int pre, const AxisPlan& P, const Fields<float>& f, cpx<float>* S,
                      const cpx<float>* tw, long long nlines, long long scs,
                      const MatView<float>& mat, Scalars* sc, const OpArgs& args,
                      double* partials, cudaStream_t st, const ReqDesc<float>* reqs, int nreq);
void pair_line_inv_f32(int D, int post, const AxisPlan& P, const cpx<float>* S,
                       const Fields<float>& f, const cpx<float>* tw, long long nlines,
                       long long scs, const MatView<float>& mat, Scalars* sc, const OpArgs& args,
                       double* partials, unsigned* counter, int negate, cudaStream_t st,
                       const ReqDesc<float>* reqs, int nreq);

// Conjugate gradients in potential coordinates for the FP32 inner solves (pcg_pot.cuh), on
// 3-D grids whose three axes have specialised two-stage plans: the axis-0 inverse with the
// direction update (mode POT_STEP) or of the iterate (POT_FIELD), the fused line pass (returns
// its CTA count, the partials of (p, K p)), and the axis-0 forward with the vector update
// (POT_UPDATE) or the right-hand side (POT_INIT)
void pot_inv_f32(int mode, const AxisPlan& P, cpx<float>* S, const cpx<float>* tw,
                 const ProjGeom& pg, const PotVecs<float>& V, const Scalars* sc, cudaStream_t st,
                 const ReqDesc<float>* reqs, int nreq);
void pot_fwd_f32(int mode, const AxisPlan& P, const cpx<float>* S, const cpx<float>* tw,
                 const ProjGeom& pg, const PotVecs<float>& V, Scalars* sc, double* partials,
                 unsigned* counter, cudaStream_t st, const ReqDesc<float>* reqs, int nreq);
int pot_line_f32(const AxisPlan& P, cpx<float>* S, const cpx<float>* tw, long long nlines,
                 long long scs, const MatView<float>& mat, Scalars* sc, double* partials,
                 cudaStream_t st, const ReqDesc<float>* reqs, int nreq);

long long& launch_counter();
int dynamic_smem_cap();

// Launch of a pass kernel with a programmatic dependency on the kernel before it on the stream
// (its CTAs may be scheduled while that one drains; the kernel itself waits in
// wait_prior_grid before touching global memory). On the legacy default stream, which such
// launches are not used on, a plain launch.
template <typename... KArgs, typename... Args>
inline void launch_pass(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                        cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = st != nullptr ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}

// Optional per-pass event timing (hom_profile_enable): kinds of launches
enum PassKind { KIND_LINE_FWD = 0, KIND_STRIDED = 1, KIND_PROJ = 2, KIND_LINE_INV = 3,
                KIND_VECTOR = 4, KIND_POT_INV = 5, KIND_POT_LINE = 6, KIND_POT_FWD = 7,
                KIND_COUNT = 8 };
bool profiling();
void prof_mark(int kind, cudaStream_t st, bool start);

}  // namespace hom
