// Internal definitions shared by the host translation units of libhom (hom_api.cu,
// hom_serve.cu): launch planning, the per-precision engine, the problem handle and the
// solver-session helpers. Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "../../include/hom.h"
#include "ops.h"
#include "passes.cuh"

namespace hom {
namespace detail {

constexpr long long kMaxNodes = 1LL << 31;

#define HOM_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      last_cuda_error() = e_;                           \
      return e_ == cudaErrorMemoryAllocation ? HOM_ERR_OOM : HOM_ERR_CUDA; \
    }                                                   \
  } while (0)

cudaError_t& last_cuda_error();

// ---------------------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------------------
// Radix plan of one axis: the prime factors of n (all <= 31) grouped into register radices of
// at most rmax (first fit, largest factors first), as few stages as possible.
inline bool plan_axis(int n, int rmax, AxisPlan* P) {
  if (n < 3 || n > kMaxAxis || n % 2 == 0) return false;
  std::vector<int> primes;
  int rem = n;
  for (int R : {31, 29, 23, 19, 17, 13, 11, 7, 5, 3})
    while (rem % R == 0) {
      primes.push_back(R);
      rem /= R;
    }
  if (rem != 1) return false;
  std::vector<int> groups;
  for (int f : primes) {
    int best = -1;
    for (size_t gi = 0; gi < groups.size(); ++gi)
      if (groups[gi] * f <= rmax && (best < 0 || groups[gi] > groups[best])) best = (int)gi;
    if (best >= 0) groups[best] *= f;
    else groups.push_back(f);
  }
  if ((int)groups.size() > kMaxStages) return false;
  std::sort(groups.begin(), groups.end(), [](int a, int b) { return a > b; });
  P->n = n;
  P->nst = (int)groups.size();
  int p = 1;
  for (int s = 0; s < kMaxStages; ++s) {
    if (s < P->nst) {
      P->radix[s] = groups[s];
      P->pprev[s] = p;
      p *= groups[s];
    } else {
      P->radix[s] = P->pprev[s] = 0;
    }
  }
  plan_fastdivs(P);
  return true;
}

// cudaMalloc behind the allocation-failure injector of hom_debug_fail_alloc (hom_api.cu):
// HOM_OK, or HOM_ERR_OOM with *p = nullptr
int alloc(void** p, size_t bytes);

// largest register radix per precision (FP64 values take twice the registers)
template <typename T> constexpr int reg_rmax() { return sizeof(T) == 8 ? 15 : 27; }

// Stage twiddles w_j = exp(-2 pi i j / n) of an odd length n: (Re w, Im w) in FP32; in FP64
// (c, t) with w = c (1 + i t), c = Re w, t = Im w / Re w (Re w is never zero for odd n), the
// cosine-factored form that the FP64 register stages fold into their multiply-adds.
template <typename T>
std::vector<cpx<T>> twiddles(int n) {
  std::vector<cpx<T>> tw(n);
  const long double twopi = 6.283185307179586476925286766559005768L;
  for (int j = 0; j < n; ++j) {
    const long double t = -twopi * (long double)j / (long double)n;
    const long double c = cosl(t), s = sinl(t);
    tw[j].x = (T)c;
    tw[j].y = sizeof(T) == 8 ? (T)(s / c) : (T)s;
  }
  return tw;
}

// ---------------------------------------------------------------------------------------
// per-precision engine: plans, twiddles, geometry, spectrum buffer view
// ---------------------------------------------------------------------------------------
template <typename T>
struct Engine {
  PassGeom g{};
  PassGeom g1{};  // same grid, one component (Ga assembly)
  AxisPlan plan[3]{};
  cpx<T>* tw[3] = {nullptr, nullptr, nullptr};
  ProjGeom pg{};
  MatView<T> mat{};
  T* field = nullptr;  // MAT_FIELD storage in precision T
  T* table = nullptr;  // phase table in precision T
  T* rk = nullptr;     // projection table scale / k.k (pg.rk)
  bool ready = false;

  int rmax_used = 0;
  size_t budget_used = 0;
  int threads_used = 0;
  bool two_line = false;  // the 3-D scalar projection runs the two-line chain (FP32 plans)

  // plan the axes with register radices <= rmax and tiles within `budget` bytes of shared
  // memory and `threads` threads per CTA, for fields of nc components (0: D); allocates the
  // twiddle tables
  int init(int D, const int* n, const int* support, size_t budget, int rmax, int threads,
           bool allow_two_line = true, int nc = 0) {
    rmax_used = rmax;
    budget_used = budget;
    threads_used = threads;
    for (int a = 0; a < D; ++a)
      if (!plan_axis(n[a], rmax, &plan[a])) return HOM_ERR_INVALID;
    if (!Ops<T>::plan_geometry(D, n, plan, budget, threads, &g, nc)) return HOM_ERR_UNSUPPORTED;
    two_line = allow_two_line && g.NC == D && Ops<T>::two_line_ok(g, plan[0], plan[1]);
    const int nl = n[D - 1];
    g1 = g;
    while (g1.LB < 16 && Ops<T>::smem_line(nl, 1, g1.LB + 2) <= budget) g1.LB += 2;
    for (int a = 0; a < D; ++a) {
      auto tw_h = twiddles<T>(n[a]);
      if (alloc((void**)&tw[a], sizeof(cpx<T>) * n[a]) != HOM_OK) return HOM_ERR_OOM;
      if (cudaMemcpy(tw[a], tw_h.data(), sizeof(cpx<T>) * n[a], cudaMemcpyHostToDevice) != cudaSuccess)
        return HOM_ERR_CUDA;
    }
    pg.C = g.scs / n[0];
    pg.cs = g.scs;
    pg.n1 = (D == 3) ? n[1] : 1;
    pg.nh = g.nh;
    pg.fdnh = make_fastdiv(g.nh);
    for (int a = 0; a < 3; ++a) pg.hw[a] = (a < D) ? (support[a] - 1) / 2 : 0;
    pg.scale = 1.0 / (double)g.nodes;
    // scale / q for every q = k.k inside the support, divided in precision T as the projection
    // kernels would (host and device divisions are both correctly rounded)
    pg.kkmax = 0;
    for (int a = 0; a < D; ++a) pg.kkmax += pg.hw[a] * pg.hw[a];
    {
      std::vector<T> rk_h((size_t)pg.kkmax + 1);
      const T sc = (T)pg.scale;
      rk_h[0] = (T)0;
      for (int q = 1; q <= pg.kkmax; ++q) rk_h[q] = sc / (T)q;
      void* d = nullptr;
      if (alloc(&d, sizeof(T) * rk_h.size()) != HOM_OK) return HOM_ERR_OOM;
      rk = static_cast<T*>(d);
      if (cudaMemcpy(d, rk_h.data(), sizeof(T) * rk_h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return HOM_ERR_CUDA;
      pg.rk = d;
    }
    ready = true;
    return HOM_OK;
  }

  // free the twiddle tables only (re-planning keeps the coefficients)
  void release_plan() {
    for (auto& t : tw) {
      if (t) cudaFree(t);
      t = nullptr;
    }
    if (rk) cudaFree(rk);
    rk = nullptr;
    pg.rk = nullptr;
  }

  void release() {
    release_plan();
    if (field) cudaFree(field);
    field = nullptr;
    if (table) cudaFree(table);
    table = nullptr;
  }

  // forward transform of the contiguous axis and the middle axis (D = 3) up to axis 0
  // y = post( F^{-1} proj F pre(x) ): one full operator application
  void apply(int pre, int mode, int post, const Fields<T>& f, cpx<T>* S, Scalars* sc,
             const OpArgs& args, double* partials, unsigned* counter, int negate,
             cudaStream_t st) const {
    apply2(pre, mode, post, f, f, S, sc, args, partials, counter, negate, st);
  }

  // same, with separate buffer sets for the pre-operator (ff) and the post-operator (fi)
  void apply2(int pre, int mode, int post, const Fields<T>& ff, const Fields<T>& fi, cpx<T>* S,
              Scalars* sc, const OpArgs& args, double* partials, unsigned* counter, int negate,
              cudaStream_t st) const {
    Ops<T>::line_fwd(g, pre, ff, S, plan[g.D - 1], tw[g.D - 1], g.NC, mat, sc, args, st, nullptr,
                     1, partials);
    if (mode == PROJ_GAMMA && two_line) {
      Ops<T>::strided_two_line(g, 0, S, plan[1], tw[1], sc, st);
      Ops<T>::proj_two_line(g, S, plan[0], tw[0], pg, sc, st);
      Ops<T>::strided_two_line(g, 1, S, plan[1], tw[1], sc, st);
    } else {
      if (g.D == 3) Ops<T>::strided(g, 1, 0, S, plan[1], tw[1], g.NC, sc, st);
      Ops<T>::proj(g, mode, S, plan[0], tw[0], pg, sc, st);
      if (g.D == 3) Ops<T>::strided(g, 1, 1, S, plan[1], tw[1], g.NC, sc, st);
    }
    Ops<T>::line_inv(g, post, S, fi, plan[g.D - 1], tw[g.D - 1], g.NC, mat, sc, args, partials,
                     counter, negate, st);
  }

  // Conjugate gradients in potential coordinates (pcg_pot.cuh) for the FP32 inner solves:
  // available for 3-D vector fields with specialised two-stage plans on all three axes
  bool pot_ok() const {
    if constexpr (sizeof(T) == 4)
      return g.D == 3 && g.NC == 3 && Ops<T>::two_line_ok(g, plan[0], plan[1]) &&
             pair_plan_f32(plan[2]);
    return false;
  }
  // the right-hand side D* x of a real field x in potential coordinates (r), u = p = 0 and
  // (r, M^{-1} r) into sc (nb, rr)
  void pot_init(const T* x, const PotVecs<T>& V, cpx<T>* S, Scalars* sc, double* partials,
                unsigned* counter, cudaStream_t st) const {
    if constexpr (sizeof(T) == 4) {
      Fields<T> f{};
      f.xin = x;
      f.cs = g.nodes;
      OpArgs args{};
      Ops<T>::line_fwd(g, PRE_IDENT, f, S, plan[2], tw[2], 3, mat, nullptr, args, st);
      Ops<T>::strided_two_line(g, 0, S, plan[1], tw[1], nullptr, st);
      pot_fwd_f32(POT_INIT, plan[0], S, tw[0], pg, V, sc, partials, counter, st, nullptr, 1);
      ++launch_counter();
    }
  }
  // one CG (or, with cheb, Chebyshev) step in potential coordinates (several requests with
  // reqs / n); Chebyshev's step length comes from its recurrence, not from (p, K p)
  void pot_step(const PotVecs<T>& V, cpx<T>* S, Scalars* sc, double* partials, unsigned* counter,
                cudaStream_t st, const ReqDesc<T>* reqs = nullptr, int n = 1,
                bool cheb = false) const {
    if constexpr (sizeof(T) == 4) {
      pot_inv_f32(POT_STEP, plan[0], S, tw[0], pg, V, sc, st, reqs, n);
      Ops<T>::strided_two_line(g, 1, S, plan[1], tw[1], sc, st, reqs, n);
      const int nb = pot_line_f32(plan[2], S, tw[2], g.nlines, g.scs, mat, sc, partials, st,
                                  reqs, n);
      ++launch_counter();
      if (!cheb) Ops<T>::cg_alpha(partials, nb, g.nodes, sc, st, reqs, n);
      Ops<T>::strided_two_line(g, 0, S, plan[1], tw[1], sc, st, reqs, n);
      pot_fwd_f32(POT_UPDATE, plan[0], S, tw[0], pg, V, sc, partials, counter, st, reqs, n);
      launch_counter() += 2;
    }
  }
  // the field x = D u of the iterate (three real components into out); sc holds the last
  // step's alpha, whose update of u the kernels defer
  void pot_field(const PotVecs<T>& V, cpx<T>* S, const Scalars* sc, T* out,
                 cudaStream_t st) const {
    if constexpr (sizeof(T) == 4) {
      pot_inv_f32(POT_FIELD, plan[0], S, tw[0], pg, V, sc, st, nullptr, 1);
      ++launch_counter();
      Ops<T>::strided_two_line(g, 1, S, plan[1], tw[1], nullptr, st);
      Fields<T> f{};
      f.out = out;
      f.cs = g.nodes;
      OpArgs args{};
      Ops<T>::line_inv(g, POST_STORE, S, f, plan[2], tw[2], 3, mat, nullptr, args, nullptr,
                       nullptr, 0, st);
    }
  }

  // one batched application over the requests of `reqs` (device array of n descriptors that
  // supply buffers, coefficients, scalars and partials); geometry and plans are shared
  void apply_batch(int pre, int mode, int post, const ReqDesc<T>* reqs, int n,
                   cudaStream_t st) const {
    Fields<T> f{};
    OpArgs args{};
    Ops<T>::line_fwd(g, pre, f, nullptr, plan[g.D - 1], tw[g.D - 1], g.NC, mat, nullptr, args, st,
                     reqs, n);
    if (mode == PROJ_GAMMA && two_line) {
      Ops<T>::strided_two_line(g, 0, nullptr, plan[1], tw[1], nullptr, st, reqs, n);
      Ops<T>::proj_two_line(g, nullptr, plan[0], tw[0], pg, nullptr, st, reqs, n);
      Ops<T>::strided_two_line(g, 1, nullptr, plan[1], tw[1], nullptr, st, reqs, n);
    } else {
      if (g.D == 3) Ops<T>::strided(g, 1, 0, nullptr, plan[1], tw[1], g.NC, nullptr, st, reqs, n);
      Ops<T>::proj(g, mode, nullptr, plan[0], tw[0], pg, nullptr, st, reqs, n);
      if (g.D == 3) Ops<T>::strided(g, 1, 1, nullptr, plan[1], tw[1], g.NC, nullptr, st, reqs, n);
    }
    Ops<T>::line_inv(g, post, nullptr, f, plan[g.D - 1], tw[g.D - 1], g.NC, mat, nullptr, args,
                     nullptr, nullptr, 0, st, reqs, n);
  }

  // plain forward transform (no projection) of ncomp (1 or NC) components, result is the
  // unscaled half spectrum
  void forward(const T* x, cpx<T>* S, int ncomp, cudaStream_t st) const {
    const PassGeom& gg = (ncomp == 1) ? g1 : g;
    Fields<T> f{};
    f.xin = x;
    f.cs = g.nodes;
    OpArgs args{};
    Ops<T>::line_fwd(gg, PRE_IDENT, f, S, plan[g.D - 1], tw[g.D - 1], ncomp, mat, nullptr, args, st);
    if (g.D == 3) Ops<T>::strided(gg, 1, 0, S, plan[1], tw[1], ncomp, nullptr, st);
    Ops<T>::strided(gg, 0, 0, S, plan[0], tw[0], ncomp, nullptr, st);
  }

  // plain inverse transform (no scaling) of a half spectrum into real fields
  void inverse(cpx<T>* S, T* y, int ncomp, cudaStream_t st) const {
    const PassGeom& gg = (ncomp == 1) ? g1 : g;
    Ops<T>::strided(gg, 0, 1, S, plan[0], tw[0], ncomp, nullptr, st);
    if (g.D == 3) Ops<T>::strided(gg, 1, 1, S, plan[1], tw[1], ncomp, nullptr, st);
    Fields<T> f{};
    f.out = y;
    f.cs = g.nodes;
    OpArgs args{};
    Ops<T>::line_inv(gg, POST_STORE, S, f, plan[g.D - 1], tw[g.D - 1], ncomp, mat, nullptr, args,
                     nullptr, nullptr, 0, st);
  }
};

// launch plan of a grid: register radix limit and shared-memory budget per CTA. Defaults, or
// what hom_autotune measured fastest for the same grid and precision in this process.
struct PlanChoice {
  int rmax;
  size_t budget;
  int threads;    // threads per CTA of the runtime-radix passes
  bool two_line;  // FP32 3-D scalar projection: two-line chain where the plans allow it
};
PlanChoice plan_choice(int precision_bytes, int d, const int* M, const int* N, int nc = 0);
int check_last();
bool spd_eigs(const double* t, int d, double* lo, double* hi);  // d <= kMaxComp

}  // namespace detail
}  // namespace hom

// entries of the per-iteration history a solve keeps at most (8 MiB of doubles)
constexpr int kHistMax = 1 << 20;

struct SolveState {
  bool active = false;
  bool solver_begun = false;  // the FP64 scalars (and history) belong to this solve
  int solver = 0;
  int stop = 0;
  bool fixed = false;
  int maxit = 0;
  int check = 8;
  int issued = 0;
  int matvecs = 0;
  double E[hom::kMaxComp] = {0, 0, 0, 0, 0, 0};
  double nE = 0;
  // iterative refinement (HOM_FP32_REFINED): FP32 inner solves of C d = r, FP64 outer residual
  bool refined = false;
  double tol = 0;
  double inner_tol = 1e-4;
  int inner_maxit = 10000;
  int outer_it = 0;
  int inner_total = 0;
  double nb = 0;         // ||b|| (FP64)
  double res = 0;        // ||b - C x|| (FP64) after the last outer update
  std::vector<double> outer_hist;  // res after each outer update
  bool finished = false;
  bool converged = false;
  float inner_ms = 0;
  int out_flags = 0;  // hom_opts.out_flags of the session
  bool pot = false;   // the FP32 inner CG runs in potential coordinates (pcg_pot.cuh)
};

struct hom_problem {
  int d = 0;
  int nc = 0;               // components of a field: d, or d (d + 1) / 2 for elasticity
  int N[3] = {1, 1, 1};     // trigonometric order
  int M[3] = {1, 1, 1};     // solve grid (N for GaNi, double grid for Ga)
  int integration = HOM_APPROX;
  int precision = HOM_FP64;
  int device = 0;
  cudaStream_t stream = nullptr;
  long long nodes = 0;
  double cA = 0, CA = 0;

  // coefficients
  int mat_kind = hom::MAT_PHASE_ISO;
  void* d_phase = nullptr;
  int index_bytes = 1;
  double* d_table = nullptr;
  double* d_inv = nullptr;        // elasticity: (C_p + omega I)^{-1} per phase (Eyre-Milton)
  double inv_omega = 0;           // the omega d_inv was formed with
  int nphase = 0;

  hom::detail::Engine<double> e64;
  hom::detail::Engine<float> e32;
  // exact integration: engine of the N grid, its half spectrum and an N-grid field, created by
  // the first hom_restrict (or HOM_OUT_NGRID output)
  hom::detail::Engine<double> eN;
  void* SN = nullptr;
  double* yN = nullptr;

  // buffers
  void* S = nullptr;              // half spectrum work buffer (sized for FP64, d components)
  size_t S_bytes = 0;
  double* vbase = nullptr;        // one allocation of 5 d |grid| doubles
  double* vec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // d x |grid| each
  float* fvec[4] = {nullptr, nullptr, nullptr, nullptr};           // FP32 inner solves
  double* partials = nullptr;
  double* d_hist = nullptr;  // per-iteration history of the FP64 solvers
  int hist_alloc = 0;
  size_t npartials = 0;
  unsigned* counter = nullptr;
  hom::Scalars* d_sc = nullptr;        // solver scalars
  hom::Scalars* d_aux = nullptr;       // scalars of auxiliary evaluations (energy, true residual)
  hom::Scalars* d_sc2 = nullptr;       // scalars of the FP32 inner solves (refinement)
  hom::Scalars* h_sc = nullptr;        // pinned host mirror
  int red_grid = 0;               // grid of the reduction kernels
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SolveState sv;
};

namespace hom {
namespace detail {

template <typename T>
MatView<T> make_view(const hom_problem* P, const T* field, const T* table) {
  MatView<T> m{};
  m.kind = P->mat_kind;
  m.nphase = P->mat_kind == MAT_FIELD ? 0 : P->nphase;
  m.ph8 = (P->mat_kind != MAT_FIELD && P->index_bytes == 1) ? (const uint8_t*)P->d_phase : nullptr;
  m.ph16 = (P->mat_kind != MAT_FIELD && P->index_bytes == 2) ? (const uint16_t*)P->d_phase : nullptr;
  m.table = table;
  m.field = field;
  return m;
}


// solver sessions (hom_api.cu)
int poll(hom_problem* P, Scalars* dst);
int upload_scalars(hom_problem* P, Scalars* dst, const Scalars& s);
int energy_eval(hom_problem* P, const double* E, const double* x, double* en, double* flux);
double true_residual(hom_problem* P, const double* E, const double* x, double* y);
int solve_stop_mode(int solver, int stop);
void enqueue_step(hom_problem* P);
void refine_enqueue_inner(hom_problem* P);
int refine_outer_update(hom_problem* P);

}  // namespace detail
}  // namespace hom
