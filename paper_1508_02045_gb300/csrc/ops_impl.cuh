// Template bodies of the launchers declared in ops.h (included by ops_f64.cu / ops_f32.cu).
#pragma once
#include <cmath>
#include <vector>
#include <type_traits>

#include "ops.h"
#include "passes.cuh"

namespace hom {

// FP32 plans with compile-time kernels (ops_pair_f32.cu); always false for FP64
template <typename T>
static bool pair_plan(const AxisPlan& P) {
  if constexpr (std::is_same<T, float>::value) return pair_plan_f32(P);
  return false;
}


// every radix of plan P at most 9: the FP64 kernels of the CG step and of hom_apply then run
// their variant without an out-of-line radix path
static bool small_radices(const AxisPlan& P) {
  for (int s = 0; s < P.nst; ++s)
    if (P.radix[s] > 9) return false;
  return true;
}

template <typename T>
cudaError_t Ops<T>::upload_constants() {
  return upload_reg_tables();
}

template <typename T>
size_t Ops<T>::smem_line(int n, int ncomp, int LB) {
  const size_t nlc = (size_t)ncomp * (LB / 2);
  return sizeof(cpx<T>) * ((size_t)n + nlc * n + nlc * (n + 1));
}
template <typename T>
size_t Ops<T>::smem_strided(int n, int TCp, int nst) {
  // twiddles + the stage buffers between the first and the last stage
  const size_t nbuf = nst >= 3 ? 2 : (nst == 2 ? 1 : 0);
  return sizeof(cpx<T>) * ((size_t)n + nbuf * (size_t)n * TCp);
}
template <typename T>
size_t Ops<T>::smem_proj(int n, int D, int TCp, int nst) {
  const size_t nbuf = nst >= 2 ? 2 : 1;
  return sizeof(cpx<T>) * ((size_t)n + nbuf * (size_t)D * n * TCp);
}

template <typename T>
size_t Ops<T>::smem_proj_scalar(int n, int TCp) {
  return sizeof(cpx<T>) * ((size_t)n + 2 * 2 * (size_t)n * TCp);
}

// Columns per CTA of a column kernel (a power of two <= tcmax, pitch TC + 1) and its threads:
// the widest tile whose first-stage butterflies (lines x TC x n / R_0) fit the thread limit and
// whose shared memory fits the budget, but at least one 32-byte sector of every row (unless
// the device limit forces narrower tiles). Threads:
// one per butterfly, rounded up to whole warps and to a multiple of TC, at most kColThreads.
enum ColKind { COL_STRIDED = 0, COL_PROJ = 1, COL_PROJ_SCALAR = 2 };

template <typename T>
static void pick_cols(const AxisPlan& P, int lines, int tcmax, size_t budget, int kind, int D,
                      int ncap, int* TC, int* TCp, int* NT) {
  const int m1 = P.n / P.radix[0];
  const int tcmin = std::max(1, 32 / (int)sizeof(cpx<T>));
  auto smem = [&](int t) {
    return kind == COL_PROJ ? Ops<T>::smem_proj(P.n, D, t + 1, P.nst)
         : kind == COL_PROJ_SCALAR ? Ops<T>::smem_proj_scalar(P.n, t + 1)
                                   : Ops<T>::smem_strided(P.n, t + 1, P.nst);
  };
  int tc = tcmax;
  while (tc > tcmin && ((long long)lines * tc * m1 > ncap || smem(tc) > budget)) tc /= 2;
  // long axes: narrower tiles rather than none at all
  while (tc > 1 && smem(tc) > (size_t)dynamic_smem_cap()) tc /= 2;
  *TC = tc;
  *TCp = tc + 1;
  const int unit = std::max(32, tc);
  const long long items = (long long)lines * tc * m1;
  *NT = (int)std::min<long long>(std::max(ncap / unit, 1) * unit, (items + unit - 1) / unit * unit);
}

template <typename T>
bool Ops<T>::plan_geometry(int D, const int* n, const AxisPlan* plan, size_t budget,
                           int threads, PassGeom* g, int nc) {
  if (threads < 32 || threads > kColThreads<T> || threads % 32) return false;
  const int NC = nc > 0 ? nc : D;
  if (NC != D && NC != D * (D + 1) / 2) return false;
  g->NTl = threads;
  g->D = D;
  g->NC = NC;
  g->nodes = 1;
  for (int a = 0; a < D; ++a) {
    g->n[a] = n[a];
    g->nodes *= n[a];
  }
  for (int a = D; a < 3; ++a) g->n[a] = 1;
  const int nl = n[D - 1];
  g->nh = (nl + 1) / 2;
  g->nlines = g->nodes / nl;
  g->scs = g->nlines * g->nh;
  g->LB = 16;
  while (g->LB > 2 && smem_line(nl, NC, g->LB) > budget) g->LB -= 2;
  if (D == 3)
    pick_cols<T>(plan[1], 1, 64, budget, COL_STRIDED, NC, threads, &g->TC1, &g->TC1p, &g->NT1);
  pick_cols<T>(plan[0], NC, 32, budget, COL_PROJ, NC, threads, &g->TC0, &g->TC0p, &g->NT0);
  pick_cols<T>(plan[0], 2, 32, budget, COL_PROJ_SCALAR, D, threads, &g->TCq, &g->TCqp, &g->NTq);
  pick_cols<T>(plan[0], 1, 64, budget, COL_STRIDED, NC, threads, &g->TCs0, &g->TCs0p, &g->NTs0);
  // the column kernels address the NC component tiles with 32-bit offsets
  if ((long long)NC * g->scs >= (1LL << 31)) return false;
  const size_t cap = (size_t)dynamic_smem_cap();
  return smem_line(nl, NC, g->LB) <= cap &&
         (NC != D || smem_proj(n[0], NC, g->TC0p, plan[0].nst) <= cap) &&
         smem_proj_scalar(n[0], g->TCqp) <= cap &&
         (D != 3 || smem_strided(n[1], g->TC1p, plan[1].nst) <= cap) &&
         smem_strided(n[0], g->TCs0p, plan[0].nst) <= cap;
}

// Opt-in shared memory per CTA minus room for the kernels' static shared variables.
inline int dynamic_smem_cap_query() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return optin - 1024;
}

#define HOM_SET_SMEM(kern)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                          cap);                                               \
    if (e_ != cudaSuccess) return e_;                                                         \
  } while (0)

template <typename T>
cudaError_t Ops<T>::prepare(int) {
  const int cap = dynamic_smem_cap_query();
  HOM_SET_SMEM((k_line_fwd<T, 2, PRE_AFFINE>));
  HOM_SET_SMEM((k_line_fwd<T, 2, PRE_LINEAR>));
  HOM_SET_SMEM((k_line_fwd<T, 2, PRE_CG>));
  HOM_SET_SMEM((k_line_fwd<T, 2, PRE_EM>));
  HOM_SET_SMEM((k_line_fwd<T, 2, PRE_IDENT>));
  HOM_SET_SMEM((k_line_fwd<T, 3, PRE_AFFINE>));
  HOM_SET_SMEM((k_line_fwd<T, 3, PRE_LINEAR>));
  HOM_SET_SMEM((k_line_fwd<T, 3, PRE_CG>));
  HOM_SET_SMEM((k_line_fwd<T, 3, PRE_EM>));
  HOM_SET_SMEM((k_line_fwd<T, 3, PRE_IDENT>));
  HOM_SET_SMEM((k_strided<T>));
  HOM_SET_SMEM((k_proj<T, 2, 2, PROJ_GAMMA>));
  HOM_SET_SMEM((k_proj<T, 2, 2, PROJ_EM>));
  HOM_SET_SMEM((k_proj<T, 3, 3, PROJ_GAMMA>));
  HOM_SET_SMEM((k_proj<T, 3, 3, PROJ_EM>));
  HOM_SET_SMEM((k_proj_scalar<T>));
  HOM_SET_SMEM((k_line_inv<T, 2, POST_STORE>));
  HOM_SET_SMEM((k_line_inv<T, 2, POST_RICH>));
  HOM_SET_SMEM((k_line_inv<T, 2, POST_CG>));
  HOM_SET_SMEM((k_line_inv<T, 2, POST_CHEB>));
  HOM_SET_SMEM((k_line_inv<T, 2, POST_EM>));
  HOM_SET_SMEM((k_line_inv<T, 2, POST_ADD>));
  HOM_SET_SMEM((k_line_inv<T, 3, POST_ADD>));
  HOM_SET_SMEM((k_line_inv<T, 3, POST_STORE>));
  HOM_SET_SMEM((k_line_inv<T, 3, POST_RICH>));
  HOM_SET_SMEM((k_line_inv<T, 3, POST_CG>));
  HOM_SET_SMEM((k_line_inv<T, 3, POST_CHEB>));
  HOM_SET_SMEM((k_line_inv<T, 3, POST_EM>));
  HOM_SET_SMEM((k_line_fwd<T, 2, PRE_CG_DOT>));
  HOM_SET_SMEM((k_line_fwd<T, 3, PRE_CG_DOT>));
  HOM_SET_SMEM((k_line_inv<T, 2, POST_CG_FUSED>));
  HOM_SET_SMEM((k_line_inv<T, 3, POST_CG_FUSED>));
  if constexpr (std::is_same<T, double>::value) {
    // the variants without an out-of-line radix path (plans with radices up to 9)
    HOM_SET_SMEM((k_line_fwd<T, 3, PRE_CG_DOT, true>));
    HOM_SET_SMEM((k_line_fwd<T, 3, PRE_LINEAR, true>));
    HOM_SET_SMEM((k_line_fwd<T, 3, PRE_AFFINE, true>));
    HOM_SET_SMEM((k_line_inv<T, 3, POST_CG_FUSED, true>));
    HOM_SET_SMEM((k_line_inv<T, 3, POST_STORE, true>));
    HOM_SET_SMEM((k_strided<T, true>));
    HOM_SET_SMEM((k_proj_scalar<T, true>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_CG_DOT, true>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_LINEAR, true>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_AFFINE, true>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_CG_FUSED, true>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_STORE, true>));
  }
  {
    // elasticity: strain fields of 3 (2-D, the 3-component line kernels above) or 6
    // components (their projection pass is two strided passes around k_proj_point)
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_CG>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_CG>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_AFFINE>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_LINEAR>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_EM>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_IDENT>));
    HOM_SET_SMEM((k_line_fwd<T, 6, PRE_CG_DOT>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_STORE>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_RICH>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_CHEB>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_EM>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_ADD>));
    HOM_SET_SMEM((k_line_inv<T, 6, POST_CG_FUSED>));
  }
  if constexpr (std::is_same<T, float>::value) return pair_prepare_f32(cap);
  return cudaSuccess;
}

template <typename T, int D>
static void line_fwd_d(const PassGeom& g, int pre, const Fields<T>& f, cpx<T>* S,
                       const AxisPlan& P, const cpx<T>* tw, int ncomp, const MatView<T>& mat,
                       Scalars* sc, const OpArgs& args, cudaStream_t st,
                       const ReqDesc<T>* reqs, int nreq, double* partials) {
  const dim3 grid((unsigned)((g.nlines + g.LB - 1) / g.LB), 1, (unsigned)nreq);
  const size_t sm = Ops<T>::smem_line(P.n, ncomp, g.LB);
  const bool prof = profiling();
  if (prof) prof_mark(KIND_LINE_FWD, st, true);
#define HOM_LF(PRE_) launch_pass(k_line_fwd<T, D, PRE_>, grid, g.NTl, sm, st, f, S, P, tw, ncomp, g.nlines, g.LB, LineDiv{make_fastdiv(g.LB), make_fastdiv(g.LB / 2)}, g.scs, mat, sc, args, partials, reqs)
#define HOM_LFS(PRE_) launch_pass(k_line_fwd<T, D, PRE_, true>, grid, g.NTl, sm, st, f, S, P, tw, ncomp, g.nlines, g.LB, LineDiv{make_fastdiv(g.LB), make_fastdiv(g.LB / 2)}, g.scs, mat, sc, args, partials, reqs)
  if constexpr (std::is_same<T, double>::value && (D == 3 || D == 6)) {
    if (small_radices(P) &&
        (pre == PRE_CG_DOT || pre == PRE_LINEAR || pre == PRE_AFFINE)) {
      if (pre == PRE_CG_DOT) HOM_LFS(PRE_CG_DOT);
      else if (pre == PRE_LINEAR) HOM_LFS(PRE_LINEAR);
      else HOM_LFS(PRE_AFFINE);
      if (prof) prof_mark(KIND_LINE_FWD, st, false);
      ++launch_counter();
      return;
    }
  }
#undef HOM_LFS
  switch (pre) {
    case PRE_AFFINE: HOM_LF(PRE_AFFINE); break;
    case PRE_LINEAR: HOM_LF(PRE_LINEAR); break;
    case PRE_CG: HOM_LF(PRE_CG); break;
    case PRE_CG_DOT: HOM_LF(PRE_CG_DOT); break;
    case PRE_EM: HOM_LF(PRE_EM); break;
    default: HOM_LF(PRE_IDENT); break;
  }
#undef HOM_LF
  if (prof) prof_mark(KIND_LINE_FWD, st, false);
  ++launch_counter();
}

template <typename T>
void Ops<T>::line_fwd(const PassGeom& g, int pre, const Fields<T>& f, cpx<T>* S,
                      const AxisPlan& P, const cpx<T>* tw, int ncomp, const MatView<T>& mat,
                      Scalars* sc, const OpArgs& args, cudaStream_t st,
                      const ReqDesc<T>* reqs, int nreq, double* partials) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.D == 3 && ncomp == g.NC && pair_line_fwd_has(ncomp, pre) && pair_plan<T>(P)) {
      const bool prof = profiling();
      if (prof) prof_mark(KIND_LINE_FWD, st, true);
      const int nb = pair_line_fwd_f32(ncomp, pre, P, f, S, tw, g.nlines, g.scs, mat, sc, args,
                                       partials, st, reqs, nreq);
      ++launch_counter();
      if (pre == PRE_CG_DOT) {
        launch_pass(k_cg_alpha<T>, dim3(1, 1, (unsigned)nreq), kThreads, 0, st, partials, nb,
                                                                      g.nodes, sc, reqs);
        ++launch_counter();
      }
      if (prof) prof_mark(KIND_LINE_FWD, st, false);
      return;
    }
  }
  if (ncomp > 3) {  // six-component strains (elasticity)
    line_fwd_d<T, 6>(g, pre, f, S, P, tw, ncomp, mat, sc, args, st, reqs, nreq, partials);
  } else if (g.D == 2 && ncomp <= 2) {
    line_fwd_d<T, 2>(g, pre, f, S, P, tw, ncomp, mat, sc, args, st, reqs, nreq, partials);
  } else {
    line_fwd_d<T, 3>(g, pre, f, S, P, tw, ncomp, mat, sc, args, st, reqs, nreq, partials);
  }
  if (pre == PRE_CG_DOT) {
    const int nb = (int)((g.nlines + g.LB - 1) / g.LB);
    launch_pass(k_cg_alpha<T>, dim3(1, 1, (unsigned)nreq), kThreads, 0, st, partials, nb, g.nodes, sc,
                                                                  reqs);
    ++launch_counter();
  }
}

template <typename T>
void Ops<T>::strided(const PassGeom& g, int axis, int inv, cpx<T>* S, const AxisPlan& P,
                     const cpx<T>* tw, int ncomp, const Scalars* sc, cudaStream_t st,
                     const ReqDesc<T>* reqs, int nreq) {
  long long C, es, bs;
  int batches, TC, TCp, NT;
  if (g.D == 3 && axis == 1) {
    C = g.nh;
    es = g.nh;
    bs = (long long)g.n[1] * g.nh;
    batches = ncomp * g.n[0];
    TC = g.TC1;
    TCp = g.TC1p;
    NT = g.NT1;
  } else {  // axis 0
    C = g.scs / g.n[0];
    es = C;
    bs = g.scs;
    batches = ncomp;
    TC = g.TCs0;
    TCp = g.TCs0p;
    NT = g.NTs0;
  }
  const bool prof = profiling();
  if (prof) prof_mark(KIND_STRIDED, st, true);
  if (pair_plan<T>(P)) {
    if constexpr (std::is_same<T, float>::value)
      pair_strided_f32(P, inv, S, tw, C, es, bs, batches, sc, st, reqs, nreq);
  } else {
    const dim3 grid((unsigned)((C + TC - 1) / TC), (unsigned)batches, (unsigned)nreq);
    const size_t sm = smem_strided(P.n, TCp, P.nst);
    bool done = false;
    if constexpr (std::is_same<T, double>::value) {
      if (small_radices(P)) {
        launch_pass(k_strided<T, true>, grid, NT, sm, st, S, P, tw, C, es, bs, TC, TCp, inv, sc,
                    reqs);
        done = true;
      }
    }
    if (!done)
      launch_pass(k_strided<T>, grid, NT, sm, st, S, P, tw, C, es, bs, TC, TCp, inv, sc, reqs);
  }
  if (prof) prof_mark(KIND_STRIDED, st, false);
  ++launch_counter();
}

template <typename T>
void Ops<T>::proj(const PassGeom& g, int mode, cpx<T>* S, const AxisPlan& P, const cpx<T>* tw,
                  const ProjGeom& pg, const Scalars* sc, cudaStream_t st,
                  const ReqDesc<T>* reqs, int nreq) {
  const bool prof = profiling();
  if (prof) prof_mark(KIND_PROJ, st, true);
  if (g.NC != g.D) {  // symmetric strain fields (elasticity)
    // the axis-0 transforms of the NC components as column passes (one CTA per component
    // tile, the tile shared memory of the strided pass), the strain projection node by node
    // between them: a one-kernel pass would hold all NC component tiles of its columns in
    // shared memory and run one CTA per SM
    const long long C = g.scs / g.n[0];
    const dim3 gs((unsigned)((C + g.TCs0 - 1) / g.TCs0), (unsigned)g.NC, (unsigned)nreq);
    const size_t sms = smem_strided(P.n, g.TCs0p, P.nst);
    // a column pass of the NC components along axis 0 (compile-time kernels for the FP32
    // plans that have them)
    auto axis0 = [&](int inv) {
      if constexpr (std::is_same<T, float>::value) {
        if (pair_plan<T>(P)) {
          pair_strided_f32(P, inv, S, tw, C, C, g.scs, g.NC, sc, st, reqs, nreq);
          return;
        }
      } else {
        if (small_radices(P)) {
          launch_pass(k_strided<T, true>, gs, g.NTs0, sms, st, S, P, tw, C, C, g.scs, g.TCs0,
                      g.TCs0p, inv, sc, reqs);
          return;
        }
      }
      launch_pass(k_strided<T>, gs, g.NTs0, sms, st, S, P, tw, C, C, g.scs, g.TCs0, g.TCs0p,
                  inv, sc, reqs);
    };
    axis0(0);
    const dim3 gp((unsigned)((pg.C + kThreads - 1) / kThreads), (unsigned)P.n, (unsigned)nreq);
#define HOM_PJE(D_, NC_, M_) launch_pass(k_proj_point<T, D_, NC_, M_>, gp, kThreads, 0, st, S, pg, P.n, (T)g.nodes, sc, reqs)
    if (g.D == 2) {
      if (mode == PROJ_EM) HOM_PJE(2, 3, PROJ_EM); else HOM_PJE(2, 3, PROJ_GAMMA);
    } else {
      if (mode == PROJ_EM) HOM_PJE(3, 6, PROJ_EM); else HOM_PJE(3, 6, PROJ_GAMMA);
    }
#undef HOM_PJE
    axis0(1);
    if (prof) prof_mark(KIND_PROJ, st, false);
    launch_counter() += 3;
    return;
  }
  if (pair_plan<T>(P)) {
    if constexpr (std::is_same<T, float>::value)
      pair_proj_f32(g.D, mode, false, P, S, tw, pg, sc, st, reqs, nreq);
    if (prof) prof_mark(KIND_PROJ, st, false);
    ++launch_counter();
    return;
  }
  if (g.D == 3 && mode == PROJ_GAMMA) {
    const dim3 grid((unsigned)((pg.C + g.TCq - 1) / g.TCq), 1, (unsigned)nreq);
    const size_t sm = smem_proj_scalar(P.n, g.TCqp);
    bool done = false;
    if constexpr (std::is_same<T, double>::value) {
      if (small_radices(P)) {
        launch_pass(k_proj_scalar<T, true>, grid, g.NTq, sm, st, S, P, tw, pg, g.TCq, g.TCqp, sc,
                    reqs);
        done = true;
      }
    }
    if (!done)
      launch_pass(k_proj_scalar<T>, grid, g.NTq, sm, st, S, P, tw, pg, g.TCq, g.TCqp, sc, reqs);
    if (prof) prof_mark(KIND_PROJ, st, false);
    ++launch_counter();
    return;
  }
  const dim3 grid((unsigned)((pg.C + g.TC0 - 1) / g.TC0), 1, (unsigned)nreq);
  const size_t sm = smem_proj(P.n, g.D, g.TC0p, P.nst);
#define HOM_PJ(D_, M_) launch_pass(k_proj<T, D_, D_, M_>, grid, g.NT0, sm, st, S, P, tw, pg, g.TC0, g.TC0p, sc, reqs)
  if (g.D == 2) {
    if (mode == PROJ_EM) HOM_PJ(2, PROJ_EM); else HOM_PJ(2, PROJ_GAMMA);
  } else {
    if (mode == PROJ_EM) HOM_PJ(3, PROJ_EM); else HOM_PJ(3, PROJ_GAMMA);
  }
#undef HOM_PJ
  if (prof) prof_mark(KIND_PROJ, st, false);
  ++launch_counter();
}

template <typename T>
bool Ops<T>::two_line_ok(const PassGeom& g, const AxisPlan& P0, const AxisPlan& P1) {
  return std::is_same<T, float>::value && g.D == 3 && pair_plan<T>(P0) && pair_plan<T>(P1);
}

// axis-1 pass of the two-line chain: component 0 by the plain pass over its n0 planes,
// components 1 and 2 together (one profiled pass)
template <typename T>
void Ops<T>::strided_two_line(const PassGeom& g, int inv, cpx<T>* S, const AxisPlan& P,
                              const cpx<T>* tw, const Scalars* sc, cudaStream_t st,
                              const ReqDesc<T>* reqs, int nreq) {
  if constexpr (std::is_same<T, float>::value) {
    const bool prof = profiling();
    if (prof) prof_mark(KIND_STRIDED, st, true);
    const long long C = g.nh, es = g.nh, bs = (long long)g.n[1] * g.nh;
    pair_strided_f32(P, inv, S, tw, C, es, bs, g.n[0], sc, st, reqs, nreq);
    pair_strided2_f32(P, inv, S, tw, C, es, bs, g.scs, g.n[0], sc, st, reqs, nreq);
    if (prof) prof_mark(KIND_STRIDED, st, false);
    launch_counter() += 2;
  }
}

template <typename T>
void Ops<T>::proj_two_line(const PassGeom& g, cpx<T>* S, const AxisPlan& P, const cpx<T>* tw,
                           const ProjGeom& pg, const Scalars* sc, cudaStream_t st,
                           const ReqDesc<T>* reqs, int nreq) {
  if constexpr (std::is_same<T, float>::value) {
    const bool prof = profiling();
    if (prof) prof_mark(KIND_PROJ, st, true);
    pair_proj_f32(g.D, PROJ_GAMMA, true, P, S, tw, pg, sc, st, reqs, nreq);
    if (prof) prof_mark(KIND_PROJ, st, false);
    ++launch_counter();
  }
}

template <typename T, int D>
static void line_inv_d(const PassGeom& g, int post, const cpx<T>* S, const Fields<T>& f,
                       const AxisPlan& P, const cpx<T>* tw, int ncomp, const MatView<T>& mat,
                       Scalars* sc, const OpArgs& args, double* partials, unsigned* counter,
                       int negate, cudaStream_t st, const ReqDesc<T>* reqs, int nreq) {
  const dim3 grid((unsigned)((g.nlines + g.LB - 1) / g.LB), 1, (unsigned)nreq);
  const size_t sm = Ops<T>::smem_line(P.n, ncomp, g.LB);
  const bool prof = profiling();
  if (prof) prof_mark(KIND_LINE_INV, st, true);
#define HOM_LI(POST_) launch_pass(k_line_inv<T, D, POST_>, grid, g.NTl, sm, st, S, f, P, tw, ncomp, g.nlines, g.LB, LineDiv{make_fastdiv(g.LB), make_fastdiv(g.LB / 2)}, g.scs, mat, sc, args, partials, counter, negate, reqs)
#define HOM_LIS(POST_) launch_pass(k_line_inv<T, D, POST_, true>, grid, g.NTl, sm, st, S, f, P, tw, ncomp, g.nlines, g.LB, LineDiv{make_fastdiv(g.LB), make_fastdiv(g.LB / 2)}, g.scs, mat, sc, args, partials, counter, negate, reqs)
  if constexpr (std::is_same<T, double>::value && (D == 3 || D == 6)) {
    if (small_radices(P) && (post == POST_CG_FUSED || post == POST_STORE)) {
      if (post == POST_CG_FUSED) HOM_LIS(POST_CG_FUSED);
      else HOM_LIS(POST_STORE);
      if (prof) prof_mark(KIND_LINE_INV, st, false);
      ++launch_counter();
      return;
    }
  }
#undef HOM_LIS
  switch (post) {
    case POST_RICH: HOM_LI(POST_RICH); break;
    case POST_CG: HOM_LI(POST_CG); break;
    case POST_CG_FUSED: HOM_LI(POST_CG_FUSED); break;
    case POST_CHEB: HOM_LI(POST_CHEB); break;
    case POST_EM: HOM_LI(POST_EM); break;
    case POST_ADD: HOM_LI(POST_ADD); break;
    default: HOM_LI(POST_STORE); break;
  }
#undef HOM_LI
  if (prof) prof_mark(KIND_LINE_INV, st, false);
  ++launch_counter();
}

template <typename T>
void Ops<T>::line_inv(const PassGeom& g, int post, const cpx<T>* S, const Fields<T>& f,
                      const AxisPlan& P, const cpx<T>* tw, int ncomp, const MatView<T>& mat,
                      Scalars* sc, const OpArgs& args, double* partials, unsigned* counter,
                      int negate, cudaStream_t st, const ReqDesc<T>* reqs, int nreq) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.D == 3 && ncomp == g.NC && pair_line_inv_has(ncomp, post) && pair_plan<T>(P)) {
      const bool prof = profiling();
      if (prof) prof_mark(KIND_LINE_INV, st, true);
      pair_line_inv_f32(ncomp, post, P, S, f, tw, g.nlines, g.scs, mat, sc, args, partials,
                        counter, negate, st, reqs, nreq);
      if (prof) prof_mark(KIND_LINE_INV, st, false);
      ++launch_counter();
      return;
    }
  }
  if (ncomp > 3) {  // six-component strains (elasticity)
    line_inv_d<T, 6>(g, post, S, f, P, tw, ncomp, mat, sc, args, partials, counter, negate, st,
                     reqs, nreq);
  } else if (g.D == 2 && ncomp <= 2) {
    line_inv_d<T, 2>(g, post, S, f, P, tw, ncomp, mat, sc, args, partials, counter, negate, st,
                     reqs, nreq);
  } else {
    line_inv_d<T, 3>(g, post, S, f, P, tw, ncomp, mat, sc, args, partials, counter, negate, st,
                     reqs, nreq);
  }
}

template <typename T>
void Ops<T>::cg_alpha(const double* partials, int nb, long long count, Scalars* sc,
                      cudaStream_t st, const ReqDesc<T>* reqs, int nreq) {
  launch_pass(k_cg_alpha<T>, dim3(1, 1, (unsigned)nreq), kThreads, 0, st, partials, nb, count, sc,
              reqs);
  ++launch_counter();
}

template <typename T>
void Ops<T>::energy(int ncomp, const T* x, long long nodes, const MatView<T>& mat, Scalars* sc,
                    double* partials, unsigned* counter, int grid, cudaStream_t st) {
  if (ncomp == 2) k_energy<T, 2><<<grid, kThreads, 0, st>>>(x, nodes, mat, sc, partials, counter);
  else if (ncomp == 3) k_energy<T, 3><<<grid, kThreads, 0, st>>>(x, nodes, mat, sc, partials, counter);
  else
    k_energy<T, 6><<<grid, kThreads, 0, st>>>(x, nodes, mat, sc, partials, counter);
  ++launch_counter();
}

template <typename T>
void Ops<T>::fill_const(T* x, long long nodes, int d, const Scalars* sc, cudaStream_t st) {
  const long long len = nodes * d;
  const unsigned grid = (unsigned)std::min<long long>((len + kThreads - 1) / kThreads, 152 * 16);
  k_fill_const<T><<<grid, kThreads, 0, st>>>(x, nodes, d, sc);
  ++launch_counter();
}

template <typename T>
void Ops<T>::demote(const double* r64, T* r, T* p, T* x, long long len, long long nodes,
                    Scalars* sc, double* partials, unsigned* counter, int grid, cudaStream_t st) {
  const bool prof = profiling();
  if (prof) prof_mark(KIND_VECTOR, st, true);
  k_demote<T><<<grid, kThreads, 0, st>>>(r64, r, p, x, len, nodes, sc, partials, counter);
  if (prof) prof_mark(KIND_VECTOR, st, false);
  ++launch_counter();
}

template <typename T>
void Ops<T>::promote(double* x64, const T* dx, long long len, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<long long>((len + kThreads - 1) / kThreads, 152 * 16);
  const bool prof = profiling();
  if (prof) prof_mark(KIND_VECTOR, st, true);
  k_promote<T><<<grid, kThreads, 0, st>>>(x64, dx, len);
  if (prof) prof_mark(KIND_VECTOR, st, false);
  ++launch_counter();
}

template <typename T>
void Ops<T>::convert_in(const double* src, T* dst, long long len, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<long long>((len + kThreads - 1) / kThreads, 152 * 16);
  k_to_working<T><<<grid, kThreads, 0, st>>>(src, dst, len);
  ++launch_counter();
}

template <typename T>
void Ops<T>::convert_out(const T* src, double* dst, long long len, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<long long>((len + kThreads - 1) / kThreads, 152 * 16);
  k_to_double<T><<<grid, kThreads, 0, st>>>(src, dst, len);
  ++launch_counter();
}

template <typename T>
void Ops<T>::pad_spectrum(const cpx<T>* Sn, cpx<T>* Sm, int D, int n0, int n1, int nh, int m0,
                          int m1, int mh, double scale, long long nlen, long long mlen,
                          cudaStream_t st) {
  const long long len = (long long)n0 * n1 * nh * D;
  const unsigned grid = (unsigned)std::min<long long>((len + kThreads - 1) / kThreads, 152 * 16);
  k_pad_spectrum<T><<<grid, kThreads, 0, st>>>(Sn, Sm, D, n0, n1, nh, m0, m1, mh, (T)scale, nlen, mlen);
  ++launch_counter();
}

template <typename T>
void Ops<T>::crop_spectrum(const cpx<T>* Sm, cpx<T>* Sn, int D, int n0, int n1, int nh, int m0,
                           int m1, int mh, double scale, long long nlen, long long mlen,
                           cudaStream_t st) {
  const long long len = (long long)n0 * n1 * nh * D;
  const unsigned grid = (unsigned)std::min<long long>((len + kThreads - 1) / kThreads, 152 * 16);
  k_crop_spectrum<T><<<grid, kThreads, 0, st>>>(Sm, Sn, D, n0, n1, nh, m0, m1, mh, (T)scale, nlen, mlen);
  ++launch_counter();
}

}  // namespace hom
