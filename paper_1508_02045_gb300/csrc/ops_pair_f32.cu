// Launchers of the FP32 kernels specialised at compile time for two-stage plans (pair_fft.cuh),
// in a translation unit of their own so that they compile in parallel with the rest.
#include <type_traits>

#include "ops.h"
#include "pair_fft.cuh"
#include "pcg_pot.cuh"

namespace hom {

bool pair_plan_f32(const AxisPlan& P) {
  if (P.nst != 2) return false;
#define HOM_PAIR_IS(R1_, R2_) \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) return true;
  HOM_PAIR_PLANS(HOM_PAIR_IS)
#undef HOM_PAIR_IS
  return false;
}

#define HOM_SET_SMEM(kern)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                          cap);                                               \
    if (e_ != cudaSuccess) return e_;                                                         \
  } while (0)

cudaError_t pair_prepare_f32(int cap) {
  using T = float;
  // this unit's copies of the register-DFT constants
  const cudaError_t e = upload_reg_tables();
  if (e != cudaSuccess) return e;
#define HOM_PAIR_SMEM(R1_, R2_)                                 \
  HOM_SET_SMEM((k_pair_strided<T, R1_, R2_, false>));           \
  HOM_SET_SMEM((k_pair_strided<T, R1_, R2_, true>));            \
  HOM_SET_SMEM((k_pair_proj<T, 2, PROJ_GAMMA, R1_, R2_>));      \
  HOM_SET_SMEM((k_pair_proj<T, 2, PROJ_EM, R1_, R2_>));         \
  HOM_SET_SMEM((k_pair_proj<T, 3, PROJ_GAMMA, R1_, R2_>));      \
  HOM_SET_SMEM((k_pair_proj<T, 3, PROJ_EM, R1_, R2_>));         \
  HOM_SET_SMEM((k_pair_proj_scalar<T, R1_, R2_, false>));       \
  HOM_SET_SMEM((k_pair_proj_scalar<T, R1_, R2_, true>));        \
  HOM_SET_SMEM((k_pair_strided2<T, R1_, R2_, false>));          \
  HOM_SET_SMEM((k_pair_strided2<T, R1_, R2_, true>));           \
  HOM_SET_SMEM((k_pair_line_fwd<T, 3, PRE_CG, R1_, R2_>));      \
  HOM_SET_SMEM((k_pair_line_fwd<T, 3, PRE_CG_DOT, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_CG_FUSED, R1_, R2_>)); \
  HOM_SET_SMEM((k_pair_line_fwd<T, 3, PRE_LINEAR, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_CG, R1_, R2_>));     \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_CHEB, R1_, R2_>));   \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_STORE, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_fwd<T, 6, PRE_CG_DOT, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_fwd<T, 6, PRE_LINEAR, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_inv<T, 6, POST_CG_FUSED, R1_, R2_>)); \
  HOM_SET_SMEM((k_pair_line_inv<T, 6, POST_CHEB, R1_, R2_>));
  HOM_PAIR_PLANS(HOM_PAIR_SMEM)
#undef HOM_PAIR_SMEM
#define HOM_POT_SMEM(R1_, R2_)                                  \
  HOM_SET_SMEM((k_pot_inv<T, R1_, R2_, POT_STEP>));             \
  HOM_SET_SMEM((k_pot_inv<T, R1_, R2_, POT_FIELD>));            \
  HOM_SET_SMEM((k_pot_fwd<T, R1_, R2_, POT_UPDATE>));           \
  HOM_SET_SMEM((k_pot_fwd<T, R1_, R2_, POT_INIT>));             \
  HOM_SET_SMEM((k_pot_line<T, 3, R1_, R2_>));
  HOM_PAIR_PLANS(HOM_POT_SMEM)
#undef HOM_POT_SMEM
  return cudaSuccess;
}

// ---- conjugate gradients in potential coordinates (pcg_pot.cuh) ----
void pot_inv_f32(int mode, const AxisPlan& P, cpx<float>* S, const cpx<float>* tw,
                 const ProjGeom& pg, const PotVecs<float>& V, const Scalars* sc, cudaStream_t st,
                 const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const bool prof = profiling();
#define HOM_POT_INV(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pot_tc_inv<R2_>();                                             \
    const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                     \
    const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + 2 * (TC + 1)));             \
    if (prof) prof_mark(KIND_POT_INV, st, true);                                               \
    if (mode == POT_FIELD)                                                                     \
      launch_pass(k_pot_inv<T, R1_, R2_, POT_FIELD>, grid, 2 * TC * R2_, sm, st, S, tw, pg, V, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pot_inv<T, R1_, R2_, POT_STEP>, grid, 2 * TC * R2_, sm, st, S, tw, pg, V, sc, reqs); \
    if (prof) prof_mark(KIND_POT_INV, st, false);                                              \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_POT_INV)
#undef HOM_POT_INV
}

void pot_fwd_f32(int mode, const AxisPlan& P, const cpx<float>* S, const cpx<float>* tw,
                 const ProjGeom& pg, const PotVecs<float>& V, Scalars* sc, double* partials,
                 unsigned* counter, cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const bool prof = profiling();
#define HOM_POT_FWD(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pot_tc_fwd<R2_>();                                             \
    const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                     \
    const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + 2 * (TC + 1)));             \
    if (prof) prof_mark(KIND_POT_FWD, st, true);                                               \
    if (mode == POT_INIT)                                                                      \
      launch_pass(k_pot_fwd<T, R1_, R2_, POT_INIT>, grid, pot_fwd_threads<R2_>(), sm, st, S, tw, pg, V, sc, partials, counter, reqs); \
    else                                                                                       \
      launch_pass(k_pot_fwd<T, R1_, R2_, POT_UPDATE>, grid, pot_fwd_threads<R2_>(), sm, st, S, tw, pg, V, sc, partials, counter, reqs); \
    if (prof) prof_mark(KIND_POT_FWD, st, false);                                              \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_POT_FWD)
#undef HOM_POT_FWD
}

int pot_line_f32(const AxisPlan& P, cpx<float>* S, const cpx<float>* tw, long long nlines,
                 long long scs, const MatView<float>& mat, Scalars* sc, double* partials,
                 cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const bool prof = profiling();
#define HOM_POT_LINE(R1_, R2_)                                                                 \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int LB = 2 * pair_lbp<3, R2_>();                                                 \
    const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                   \
    const size_t sm = PairFwdSmem<3, R1_, R2_>::bytes;                                         \
    constexpr int NT = pair_line_threads<3, R2_>();                                            \
    if (prof) prof_mark(KIND_POT_LINE, st, true);                                              \
    launch_pass(k_pot_line<T, 3, R1_, R2_>, grid, NT, sm, st, S, tw, nlines, scs, mat, sc,       \
                partials, reqs);                                                               \
    if (prof) prof_mark(KIND_POT_LINE, st, false);                                             \
    return (int)grid.x;                                                                        \
  }
  HOM_PAIR_PLANS(HOM_POT_LINE)
#undef HOM_POT_LINE
  return 0;
}

// Shared memory requested by a strided CTA of 128 threads or more: 39424 bytes a CTA with the
// driver's reserve, so that six no longer fit the SM (228 KiB) and five keep its 196 KiB
// configuration. The 243-point forward pass, whose registers allow six CTAs, ran 0.075 instead
// of 0.078 ms (averaged with the inverse pass) at five: six CTAs queue up on shared memory.
constexpr size_t kPairStridedMinSmem = 38400;

void pair_strided_f32(const AxisPlan& P, int inv, cpx<float>* S, const cpx<float>* tw,
                      long long C, long long es, long long bs, int batches, const Scalars* sc,
                      cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
#define HOM_PAIR_ST(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pair_tc_strided<R2_>();                                                 \
    const dim3 grid((unsigned)((C + TC - 1) / TC), (unsigned)batches, (unsigned)nreq);        \
    size_t sm = sizeof(cpx<T>) * (size_t)(R1_ * R2_) * (TC + 2);                                \
    if (TC * R2_ >= 128 && sm < kPairStridedMinSmem) sm = kPairStridedMinSmem;                 \
    if (inv)                                                                                   \
      launch_pass(k_pair_strided<T, R1_, R2_, true>, grid, TC * R2_, sm, st, S, tw, C, es, bs, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pair_strided<T, R1_, R2_, false>, grid, TC * R2_, sm, st, S, tw, C, es, bs, sc, reqs); \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_ST)
#undef HOM_PAIR_ST
}

void pair_strided2_f32(const AxisPlan& P, int inv, cpx<float>* S, const cpx<float>* tw,
                       long long C, long long es, long long bs, long long cs, int planes,
                       const Scalars* sc, cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
#define HOM_PAIR_ST2(R1_, R2_)                                                                 \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pair_tc_strided<R2_>();                                                 \
    const dim3 grid((unsigned)((C + TC - 1) / TC), (unsigned)planes, (unsigned)nreq);         \
    const size_t sm = sizeof(cpx<T>) * (size_t)(R1_ * R2_) * (1 + 2 * (TC + 1));               \
    if (inv)                                                                                   \
      launch_pass(k_pair_strided2<T, R1_, R2_, true>, grid, 2 * TC * R2_, sm, st, S, tw, C, es, bs, cs, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pair_strided2<T, R1_, R2_, false>, grid, 2 * TC * R2_, sm, st, S, tw, C, es, bs, cs, sc, reqs); \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_ST2)
#undef HOM_PAIR_ST2
}

void pair_proj_f32(int D, int mode, bool two, const AxisPlan& P, cpx<float>* S,
                   const cpx<float>* tw, const ProjGeom& pg, const Scalars* sc, cudaStream_t st,
                   const ReqDesc<float>* reqs, int nreq) {
  using T = float;
#define HOM_PAIR_PJ_D(D_, R1_, R2_)                                                            \
  {                                                                                            \
    constexpr int TC = pair_tc_proj<D_, R2_>();                                                \
    const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                     \
    const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + D_ * (TC + 1)));        \
    if (mode == PROJ_EM)                                                                       \
      launch_pass(k_pair_proj<T, D_, PROJ_EM, R1_, R2_>, grid, D_ * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pair_proj<T, D_, PROJ_GAMMA, R1_, R2_>, grid, D_ * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
  }
#define HOM_PAIR_PJ(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    if (D == 2) {                                                                              \
      HOM_PAIR_PJ_D(2, R1_, R2_)                                                               \
    } else if (mode == PROJ_GAMMA) {                                                           \
      constexpr int TC = pair_tc_proj_scalar<R2_>();                                           \
      const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                   \
      const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + 2 * (TC + 1)));           \
      if (two)                                                                                 \
        launch_pass(k_pair_proj_scalar<T, R1_, R2_, true>, grid, 2 * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
      else                                                                                     \
        launch_pass(k_pair_proj_scalar<T, R1_, R2_, false>, grid, 2 * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
    } else {                                                                                   \
      HOM_PAIR_PJ_D(3, R1_, R2_)                                                               \
    }                                                                                          \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_PJ)
#undef HOM_PAIR_PJ
#undef HOM_PAIR_PJ_D
}

int pair_line_fwd_f32(int D, int pre, const AxisPlan& P, const Fields<float>& f, cpx<float>* S,
                      const cpx<float>* tw, long long nlines, long long scs,
                      const MatView<float>& mat, Scalars* sc, const OpArgs& args,
                      double* partials, cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const FastDiv fdn = make_fastdiv(P.n);
#define HOM_PAIR_LF_P(D_, PRE_, R1_, R2_)                                                      \
  launch_pass(k_pair_line_fwd<T, D_, PRE_, R1_, R2_>, grid, NT, sm, st, f, S, tw, nlines, scs, mat, sc, \
              args, fdn, partials, reqs)
#define HOM_PAIR_LF(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    if (D == 6) {                                                                              \
      constexpr int LB = 2 * pair_lbp<6, R2_>();                                               \
      const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                 \
      const size_t sm = PairFwdSmem<6, R1_, R2_>::bytes;                                       \
      constexpr int NT = pair_line_threads<6, R2_>();                                          \
      if (pre == PRE_CG_DOT) HOM_PAIR_LF_P(6, PRE_CG_DOT, R1_, R2_);                           \
      else HOM_PAIR_LF_P(6, PRE_LINEAR, R1_, R2_);                                             \
      return (int)grid.x;                                                                      \
    }                                                                                          \
    constexpr int LB = 2 * pair_lbp<3, R2_>();                                                 \
    const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                   \
    const size_t sm = PairFwdSmem<3, R1_, R2_>::bytes;                                         \
    constexpr int NT = pair_line_threads<3, R2_>();                                            \
    if (pre == PRE_CG) HOM_PAIR_LF_P(3, PRE_CG, R1_, R2_);                                     \
    else if (pre == PRE_CG_DOT) HOM_PAIR_LF_P(3, PRE_CG_DOT, R1_, R2_);                        \
    else HOM_PAIR_LF_P(3, PRE_LINEAR, R1_, R2_);                                               \
    return (int)grid.x;                                                                        \
  }
  HOM_PAIR_PLANS(HOM_PAIR_LF)
  return 0;
#undef HOM_PAIR_LF
#undef HOM_PAIR_LF_P
}

void pair_line_inv_f32(int D, int post, const AxisPlan& P, const cpx<float>* S,
                       const Fields<float>& f, const cpx<float>* tw, long long nlines,
                       long long scs, const MatView<float>& mat, Scalars* sc, const OpArgs& args,
                       double* partials, unsigned* counter, int negate, cudaStream_t st,
                       const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const FastDiv fdn = make_fastdiv(P.n);
#define HOM_PAIR_LI_P(D_, POST_, R1_, R2_)                                                     \
  launch_pass(k_pair_line_inv<T, D_, POST_, R1_, R2_>, grid, NT, sm, st, S, f, tw, nlines, scs, mat, \
              sc, args, partials, counter, negate, fdn, reqs)
#define HOM_PAIR_LI(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    if (D == 6) {                                                                              \
      constexpr int LB = 2 * pair_lbp<6, R2_>();                                               \
      const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                 \
      const size_t sm = PairFwdSmem<6, R1_, R2_>::bytes;                                       \
      constexpr int NT = pair_line_threads<6, R2_>();                                          \
      if (post == POST_CG_FUSED) HOM_PAIR_LI_P(6, POST_CG_FUSED, R1_, R2_);                    \
      else HOM_PAIR_LI_P(6, POST_CHEB, R1_, R2_);                                              \
      return;                                                                                  \
    }                                                                                          \
    constexpr int LB = 2 * pair_lbp<3, R2_>();                                                 \
    const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                   \
    const size_t sm = PairFwdSmem<3, R1_, R2_>::bytes;                                         \
    constexpr int NT = pair_line_threads<3, R2_>();                                            \
    if (post == POST_CG) HOM_PAIR_LI_P(3, POST_CG, R1_, R2_);                                  \
    else if (post == POST_CG_FUSED) HOM_PAIR_LI_P(3, POST_CG_FUSED, R1_, R2_);                 \
    else if (post == POST_CHEB) HOM_PAIR_LI_P(3, POST_CHEB, R1_, R2_);                         \
    else HOM_PAIR_LI_P(3, POST_STORE, R1_, R2_);                                               \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_LI)
#undef HOM_PAIR_LI
#undef HOM_PAIR_LI_P
}

}  // namespace hom
