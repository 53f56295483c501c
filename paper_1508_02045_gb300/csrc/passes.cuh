// The fused FFT passes of the operator e -> G A (E + e) and the solver kernels around them.
//
// A field on the solve grid (n_0, ..., n_{D-1}) has the last axis contiguous; its transform is
// stored as a half spectrum (k_{D-1} = 0 .. (n_{D-1}-1)/2, the rest follows from Hermitian
// symmetry of real fields, Section 2.1), layout [component][k_0]...[k_{D-2}][k_{D-1}].
//
// One operator application is
//   line_fwd  : pre-operator (A(E+x), A p, ...) + forward real DFT of the contiguous axis;
//               two real lines share one complex transform
//   strided   : forward DFT of the middle axis (D = 3)
//   proj      : forward DFT of axis 0, the projection Gamma^ (eq. (proj); with the truncation
//               to Z_N of eq. (discrete_proj) on a double grid; or I - 2 Gamma^ of
//               Algorithm 4), the 1/|N| of eq. (DFT), and the inverse DFT of axis 0
//   strided   : inverse DFT of the middle axis (D = 3)
//   line_inv  : inverse real DFT of the contiguous axis + the solver's post-operator (vector
//               update and inner-product partials of Algorithms 1-4).
// Reductions are deterministic: one partial per CTA, summed in a fixed order by the last CTA
// to finish, which then runs the scalar part of the algorithm step ("finisher").
#pragma once
#include "common.cuh"
#include "fft_reg.cuh"

namespace hom {

// resident CTAs per SM the pass kernels are compiled for (<= 128 registers per thread). Four
// CTAs (64 registers) were measured slower for FP32: the radix stages spill.
template <typename T>
constexpr int kMinBlocks = 2;

// thread limit of the column kernels (strided, proj): compiled, like the line kernels, for
// 128 registers a thread (a radix-27 FP32 or radix-15 FP64 butterfly held in registers); the
// stage functions they share are compiled once for that budget
template <typename T>
constexpr int kColThreads = kThreads;

// ---------------------------------------------------------------------------------------
// deterministic block reduction + last-block finisher
// ---------------------------------------------------------------------------------------
template <int NV, int MAXW = kThreads / 32>
__device__ bool reduce_and_last(double (&acc)[NV], double* partials, unsigned* counter,
                                double (&tot)[NV]) {
  __shared__ double red[NV][MAXW];
  __shared__ double fin[NV];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);  // blocks are whole warps, at most MAXW of them
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = acc[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[v][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[v][w];
      partials[(size_t)bid * NV + v] = s;
    }
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    am_last = (t == (unsigned)(nblocks - 1));
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += __ldcg(&partials[(size_t)b * NV + v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) red[v][warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double f = 0.0;
      for (int w = 0; w < nw; ++w) f += red[v][w];
      fin[v] = f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) tot[v] = fin[v];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Per-CTA partial of a grid reduction without the completion ticket: the CTA writes its sum
// and a later kernel (k_cg_alpha) adds the partials in a fixed order, so the producing kernel
// needs no fence or atomic at its end.
template <int NV>
__device__ void block_partial(double (&acc)[NV], double* partials) {
  __shared__ double redp[NV][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = acc[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) redp[v][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += redp[v][w];
      partials[(size_t)bid * NV + v] = s;
    }
  }
}

// ---------------------------------------------------------------------------------------
// coefficient products
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int phase_at(const MatView<T>& m, long long g) {
  return m.ph8 ? (int)m.ph8[g] : (int)m.ph16[g];
}

// v = A(x^g) w
template <typename T, int D>
__device__ __forceinline__ void mat_apply(const MatView<T>& m, long long g, const T (&w)[D],
                                          T (&v)[D]) {
  if (m.kind == MAT_FIELD) {
    const T a = m.field[g];
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = a * w[i];
  } else if (m.kind == MAT_PHASE_ISO) {
    const T a = __ldg(&m.table[phase_at(m, g)]);
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = a * w[i];
  } else {
    const T* t = m.table + phase_at(m, g) * D * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T s = 0;
#pragma unroll
      for (int j = 0; j < D; ++j) s = fma(__ldg(&t[i * D + j]), w[j], s);
      v[i] = s;
    }
  }
}

// the coefficient of node g in two steps, so that the loads of a batch of nodes can be issued
// before any of them is used: fetch (phase index or field value), then evaluate v = A w
// a phase index carried through a value of the working precision by its bits (a numeric
// conversion would cost two FP64-pipe instructions a node)
__device__ __forceinline__ double phase_bits(int ph, double) {
  return __longlong_as_double((long long)ph);
}
__device__ __forceinline__ float phase_bits(int ph, float) { return __int_as_float(ph); }
__device__ __forceinline__ int phase_of(double s) { return (int)__double_as_longlong(s); }
__device__ __forceinline__ int phase_of(float s) { return __float_as_int(s); }

template <typename T>
__device__ __forceinline__ T mat_fetch(const MatView<T>& m, long long g) {
  if (m.kind == MAT_FIELD) return m.field[g];
  return phase_bits(phase_at(m, g), T());
}

template <typename T, int D>
__device__ __forceinline__ void mat_eval(const MatView<T>& m, T sample, const T (&w)[D],
                                         T (&v)[D]) {
  if (m.kind == MAT_FIELD || m.kind == MAT_PHASE_ISO) {
    const T a = (m.kind == MAT_FIELD) ? sample : __ldg(&m.table[phase_of(sample)]);
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = a * w[i];
  } else {
    const T* t = m.table + phase_of(sample) * D * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T s = 0;
#pragma unroll
      for (int j = 0; j < D; ++j) s = fma(__ldg(&t[i * D + j]), w[j], s);
      v[i] = s;
    }
  }
}

// asynchronous global -> shared copies of one complex element (LDGSTS), and the wait
template <typename T>
__device__ __forceinline__ void cp_async_elem(cpx<T>* dst, const cpx<T>* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(cpx<T>) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// (A + omega I)^{-1} w with the coefficient given by a fetched sample (see mat_fetch)
template <typename T, int D>
__device__ __forceinline__ void mat_shift_solve_s(const MatView<T>& m, T sample, T omega,
                                                  const T (&w)[D], T (&v)[D]) {
  if (m.kind == MAT_FIELD || m.kind == MAT_PHASE_ISO) {
    const T a = (m.kind == MAT_FIELD) ? sample : __ldg(&m.table[phase_of(sample)]);
    const T inv = (T)1 / (a + omega);
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = w[i] * inv;
    return;
  }
  const int ph = phase_of(sample);
  if (D > 3) {  // precomputed (A_p + omega I)^{-1} of every phase
    const T* ti = m.inv + ph * D * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < D; ++j) acc = fma(__ldg(&ti[i * D + j]), w[j], acc);
      v[i] = acc;
    }
    return;
  }
  const T* t = m.table + ph * D * D;
  T M[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) M[i][j] = __ldg(&t[i * D + j]) + (i == j ? omega : (T)0);
  if (D == 2) {
    const T det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    v[0] = (M[1][1] * w[0] - M[0][1] * w[1]) / det;
    v[1] = (M[0][0] * w[1] - M[1][0] * w[0]) / det;
  } else {
    const T c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    const T c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    const T c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    const T det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
    const T c10 = M[0][2] * M[2][1] - M[0][1] * M[2][2];
    const T c11 = M[0][0] * M[2][2] - M[0][2] * M[2][0];
    const T c12 = M[0][1] * M[2][0] - M[0][0] * M[2][1];
    const T c20 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
    const T c21 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
    const T c22 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    v[0] = (c00 * w[0] + c10 * w[1] + c20 * w[2]) / det;
    v[1] = (c01 * w[0] + c11 * w[1] + c21 * w[2]) / det;
    v[2] = (c02 * w[0] + c12 * w[1] + c22 * w[2]) / det;
  }
}

// ---------------------------------------------------------------------------------------
// Buffers of one operator application / solver step
// ---------------------------------------------------------------------------------------
// Scalars of a single operator application outside a solve (Scalars pointer is then null).
struct OpArgs {
  double E[kMaxComp];
  double omega;
};

template <typename T>
struct Fields {
  const T* xin;   // operand of the pre-operator (x, or r for PRE_CG)
  T* p;           // PRE_CG / POST_CG / POST_CHEB: search direction
  T* out;         // POST_STORE: destination; POST_CG: C p
  T* x;           // POST_RICH: buffer pair base (x_a, x_b = x + d|N|); POST_CHEB / POST_EM: x
  T* r;           // POST_CHEB: residual; POST_STORE with negate: r
  long long cs;   // component stride (|N|)
};

// Per-request arguments of a batched launch (blockIdx.z selects the request): several
// same-shape problems advance through one launch per pass, each with its own buffers,
// coefficients, device scalars and reduction partials.
template <typename T>
struct ReqDesc {
  Fields<T> ff;        // pre-operator buffers (line_fwd)
  Fields<T> fi;        // post-operator buffers (line_inv)
  cpx<T>* S;           // half-spectrum work buffer
  MatView<T> mat;
  Scalars* sc;
  double* partials;
  unsigned* counter;
};

// ---------------------------------------------------------------------------------------
// line_fwd: pre-operator + forward real DFT of the contiguous axis
// ---------------------------------------------------------------------------------------
// PRE_CG_DOT: the CTA's partial of (p, A p); k_cg_alpha completes the sum
template <typename T>
__device__ __forceinline__ void line_fwd_partial_cg(const DotAcc<T>& dacc, double* partials) {
  double acc[1] = {dacc.value()};
  block_partial<1>(acc, partials);
}

// (p, A p) from the nblocks partials of the PRE_CG_DOT pass, summed in a fixed order by one
// CTA per request (blockIdx.z), and the step length alpha = (r, r) / (p, A p) of Algorithm 2,
// set before the transforms of C p run
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cg_alpha(const double* partials, int nblocks, long long count, Scalars* sc,
           const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  __shared__ double red[kThreads / 32];
  if (reqs != nullptr) {
    partials = reqs[blockIdx.z].partials;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) f += red[w];
    const double pAp = f / (double)count;
    sc->pAp = pAp;
    sc->alpha = sc->rr / pAp;
  }
}

// Pre-operator of the lines l0 .. l0 + LB - 1 (pointwise, coalesced loads in batches of K
// nodes): component a of line l0 + ll goes to the real (ll even) or imaginary (ll odd) part of
// the shared-memory complex line b0 + (a * half + ll / 2) * n, so that two real lines share one
// complex transform. RAW: component a of the tile is instead stored as it lies in the field,
// node idx of the tile at element raw[a] + idx of shared memory (the specialised FP32 line pass
// packs the line pairs when its first stage loads them).
template <typename T, int D, int PRE, int K = (sizeof(T) == 4 ? 8 : (D > 3 ? 2 : 4)), int NC = 0,
          bool RAW = false>
__device__ __forceinline__ void line_pre_to_smem(const Fields<T>& f, int b0, int n, int half,
                                                 int ncomp, long long l0, int LB, long long nlines,
                                                 FastDiv fdn, const MatView<T>& mat,
                                                 const Scalars* sc, const OpArgs& args,
                                                 DotAcc<T>* dacc = nullptr,
                                                 const int* raw = nullptr) {
  constexpr bool CG = PRE == PRE_CG || PRE == PRE_CG_DOT;
  // NC > 0: the line length as a compile-time constant (specialised kernels)
  if (NC > 0) n = NC;
  cpx<T>* sm = smem_c<T>();
  const double* Es = sc != nullptr ? sc->E : args.E;
  T E[D];
#pragma unroll
  for (int a = 0; a < D; ++a) E[a] = (T)Es[a];
  const T omega = (T)(sc != nullptr ? sc->omega : args.omega);
  const T beta = sc != nullptr ? (T)sc->beta : (T)0;
  // Richardson keeps x_m and x_{m-1} in a buffer pair; the operand is the current one
  const T* xin = f.xin;
  if (f.x != nullptr && sc != nullptr) xin = f.x + (sc->which ? D * f.cs : 0);
  // the CTA's lines are contiguous: node idx of the tile is node g0 + idx of the grid
  const long long g0 = l0 * n;
  const int ntile = LB * n;
  const int nvalid = (int)min((long long)ntile, (nlines - l0) * n);
  const T* __restrict__ xb = xin + g0;
  const T* __restrict__ pb = f.p + g0;
  T* pw = f.p + g0;
  // batches of K nodes per thread: every global load of a batch is issued before any use
  for (int base = 0; base < ntile; base += K * blockDim.x) {
    T xv[K][D], pv[K][D], ms[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int idx = base + k * blockDim.x + threadIdx.x;
      const bool ok = idx < nvalid;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        xv[k][a] = (ok && a < ncomp) ? xb[a * f.cs + idx] : (T)0;
        pv[k][a] = (CG && ok) ? pb[a * f.cs + idx] : (T)0;
      }
      ms[k] = (PRE != PRE_IDENT && ok) ? mat_fetch<T>(mat, g0 + idx) : (T)0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int idx = base + k * blockDim.x + threadIdx.x;
      if (idx >= ntile) continue;
      const bool ok = idx < nvalid;
      T v[D];
      if (PRE == PRE_IDENT) {
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = xv[k][a];
      } else {
        T w[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          if (CG) {
            w[a] = xv[k][a] + beta * pv[k][a];
            if (ok) pw[a * f.cs + idx] = w[a];
          } else {
            w[a] = xv[k][a] + (PRE == PRE_AFFINE && ok ? E[a] : (T)0);
          }
        }
        mat_eval<T, D>(mat, ms[k], w, v);
        if (PRE == PRE_EM) {
#pragma unroll
          for (int a = 0; a < D; ++a) v[a] -= omega * w[a];
        }
        if (PRE == PRE_CG_DOT && ok) {
#pragma unroll
          for (int a = 0; a < D; ++a) dacc->add(w[a], v[a]);
        }
        if (!ok) {
#pragma unroll
          for (int a = 0; a < D; ++a) v[a] = 0;
        }
      }
      if (RAW) {
        T* smt = reinterpret_cast<T*>(sm);
#pragma unroll
        for (int a = 0; a < D; ++a)
          if (a < ncomp) smt[raw[a] + idx] = v[a];
      } else {
        const int ll = NC > 0 ? idx / NC : fdiv(idx, fdn), j = idx - ll * n;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          if (a < ncomp) {
            cpx<T>& e = sm[b0 + (a * half + (ll >> 1)) * n + j];
            if (ll & 1) e.y = v[a];
            else e.x = v[a];
          }
        }
      }
    }
  }
}

template <typename T, int D, int PRE, bool SMALLR = false>
__global__ void __launch_bounds__(kThreads, SMALLR ? 3 : kMinBlocks<T>)
k_line_fwd(Fields<T> f, cpx<T>* S, AxisPlan P, const cpx<T>* __restrict__ twg,
           int ncomp, long long nlines, int LB, LineDiv ld, long long scs, MatView<T> mat,
           Scalars* sc, OpArgs args, double* partials, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  if (reqs != nullptr) {
    const ReqDesc<T>& R = reqs[blockIdx.z];
    f = R.ff;
    S = R.S;
    mat = R.mat;
    sc = R.sc;
    partials = R.partials;
  }
  if (sc != nullptr && sc->done) return;
  const int n = P.n, nh = (n + 1) / 2;
  const int half = LB / 2;
  const int nlc = ncomp * half;
  cpx<T>* sm = smem_c<T>();
  const int b0 = n, b1 = n + nlc * n;  // element offsets; twiddles at 0
  __shared__ AxisPlan Ps;
  if (threadIdx.x == 0) Ps = P;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = twg[i];
  const long long l0 = (long long)blockIdx.x * LB;
  DotAcc<T> dacc;
  line_pre_to_smem<T, D, PRE>(f, b0, n, half, ncomp, l0, LB, nlines, P.fdn, mat, sc, args, &dacc);
  __syncthreads();
  const int res = reg_lines<T, SMALLR>(b0, b1, &Ps, nlc, n, 1, false, false, 0);
  for (int idx = threadIdx.x; idx < nlc * nh; idx += blockDim.x) {
    const int lc = fdiv(idx, P.fdnh), k = idx - lc * nh;
    const int a = fdiv(lc, ld.half), pr = lc - a * half;
    const cpx<T> zk = sm[res + lc * n + k];
    const cpx<T> zm = sm[res + lc * n + (k ? n - k : 0)];
    cpx<T> A, B;
    A.x = (T)0.5 * (zk.x + zm.x);
    A.y = (T)0.5 * (zk.y - zm.y);
    B.x = (T)0.5 * (zk.y + zm.y);
    B.y = (T)-0.5 * (zk.x - zm.x);
    const long long la = l0 + 2 * pr;
    if (la < nlines) S[a * scs + la * nh + k] = A;
    if (la + 1 < nlines) S[a * scs + (la + 1) * nh + k] = B;
  }
  if (PRE == PRE_CG_DOT) line_fwd_partial_cg(dacc, partials);
}

// ---------------------------------------------------------------------------------------
// strided: DFT along a strided axis, in place; blockIdx.y = batch, blockIdx.x = column tile
// ---------------------------------------------------------------------------------------
// One CTA per tile of TC columns, one thread per first-stage butterfly (TC x n / R_0, capped at
// kColThreads): the first stage reads the rows of the tile straight from the spectrum (a warp
// takes consecutive columns, so each row segment is one coalesced access) and the last stage
// writes them back, so the tile crosses shared memory only between stages.
template <typename T, bool SMALLR = false>
__global__ void __launch_bounds__(kColThreads<T>, 2)
k_strided(cpx<T>* S, AxisPlan P, const cpx<T>* __restrict__ twg, long long C, long long es,
          long long bs, int TC, int TCp, int inv, const Scalars* sc,
          const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  const int n = P.n;
  cpx<T>* sm = smem_c<T>();
  __shared__ AxisPlan Ps;
  if (threadIdx.x == 0) Ps = P;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = twg[i];
  __syncthreads();
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, C - c0);
  const Loc<T> gl = gcols<T>(S + (long long)blockIdx.y * bs + c0, (int)es, 0, -1, ncols);
  reg_columns_global<T, SMALLR>(gl, n, n + n * TCp, TCp, 0, -1, ncols, &Ps, inv != 0);
}

// ---------------------------------------------------------------------------------------
// proj: forward DFT of axis 0, projection, inverse DFT of axis 0 (all D components)
// ---------------------------------------------------------------------------------------
struct ProjGeom {
  long long C;    // columns: product of the middle axes x half length of the last axis
  long long cs;   // component stride of the spectrum
  int n1;         // middle axis length (D = 3), 1 otherwise
  int nh;         // half length of the last axis
  FastDiv fdnh;   // division by nh
  int hw[3];      // support half-widths: keep |k_a| <= hw[a] (Z_N inside Z_M); else zero
  double scale;   // 1/|grid| of the forward transform (eq. (DFT))
  const void* rk; // scale / q for q = k.k = 0 .. kkmax in the working precision (entry 0 unused),
                  // the value the division below would give, or null (divide)
  int kkmax;      // sum of hw[a]^2
};

// scale / k.k of a frequency inside the support (kk > 0): from the table when the engine has one
// (a load instead of an FP64 division), else divided
template <typename T>
__device__ __forceinline__ T inv_kk(const ProjGeom& g, T scale, int kk) {
  return g.rk != nullptr ? __ldg(static_cast<const T*>(g.rk) + min(kk, g.kkmax)) : scale / (T)kk;
}

// Mandel storage of a symmetric D x D tensor: component m holds (i, j) = (mandel_i, mandel_j),
// off-diagonal entries scaled by sqrt 2 (D = 2: 11, 22, 12; D = 3: 11, 22, 33, 23, 13, 12)
template <int D>
__host__ __device__ constexpr int mandel_i(int m) {
  return D == 2 ? (m == 2 ? 0 : m) : (m < 3 ? m : (m == 3 ? 1 : 0));
}
template <int D>
__host__ __device__ constexpr int mandel_j(int m) {
  return D == 2 ? (m == 2 ? 1 : m) : (m < 3 ? m : (m == 5 ? 1 : 2));
}

// The projection of one frequency k (row j of a column) on the NC transformed components v:
//  NC == D (vector fields, eq. (proj)): Gamma^ v = k (k . v) / |k|^2;
//  NC == D (D + 1) / 2 (symmetric strains in Mandel storage, the elasticity form): with
//  e the tensor of v and q = e k, Gamma^ e = (k q^T + q k^T) / |k|^2 - (k.e.k) k k^T / |k|^4,
//  the orthogonal projection onto the compatible strains sym(k u^T);
// c1 = scale / |k|^2 (0 at k = 0 and outside the support); MODE PROJ_EM gives scale v - 2 Gamma^ v.
template <typename T, int D, int NC, int MODE>
__device__ __forceinline__ void proj_point(const int (&k)[3], T c1, int kk, T scale,
                                           const cpx<T> (&v)[NC], cpx<T> (&o)[NC],
                                           T nodes = (T)0) {
  if (NC == D) {
    cpx<T> kv = {0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      kv.x = fma((T)k[a], v[a].x, kv.x);
      kv.y = fma((T)k[a], v[a].y, kv.y);
    }
    kv.x *= c1;
    kv.y *= c1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (MODE == PROJ_GAMMA) {
        o[a].x = (T)k[a] * kv.x;
        o[a].y = (T)k[a] * kv.y;
      } else {  // (I - 2 Gamma^) v
        o[a].x = fma((T)(-2 * k[a]), kv.x, scale * v[a].x);
        o[a].y = fma((T)(-2 * k[a]), kv.y, scale * v[a].y);
      }
    }
  } else {
    const T r2 = (T)0.70710678118654752440;  // 1 / sqrt 2
    const T s2 = (T)1.41421356237309504880;  // sqrt 2
    // c2 = scale / |k|^4 = c1^2 |N| (c1 = scale / |k|^2, scale = 1 / |N|): no division
    const T c2 = nodes > (T)0 ? c1 * c1 * nodes : (kk > 0 ? c1 / (T)kk : (T)0);
    // q = e k
    cpx<T> q[D];
#pragma unroll
    for (int i = 0; i < D; ++i) q[i] = cpx<T>{0, 0};
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int i = mandel_i<D>(m), j = mandel_j<D>(m);
      if (i == j) {
        q[i].x = fma((T)k[i], v[m].x, q[i].x);
        q[i].y = fma((T)k[i], v[m].y, q[i].y);
      } else {
        const T ex = v[m].x * r2, ey = v[m].y * r2;
        q[i].x = fma((T)k[j], ex, q[i].x);
        q[i].y = fma((T)k[j], ey, q[i].y);
        q[j].x = fma((T)k[i], ex, q[j].x);
        q[j].y = fma((T)k[i], ey, q[j].y);
      }
    }
    cpx<T> kek = {0, 0};
#pragma unroll
    for (int i = 0; i < D; ++i) {
      kek.x = fma((T)k[i], q[i].x, kek.x);
      kek.y = fma((T)k[i], q[i].y, kek.y);
    }
    // Gamma^ e = k (x) Q + Q (x) k - S k (x) k with Q = c1 q and S = c2 (k . e . k)
    cpx<T> Q[D];
#pragma unroll
    for (int i = 0; i < D; ++i) Q[i] = cpx<T>{q[i].x * c1, q[i].y * c1};
    const cpx<T> Sk = {kek.x * c2, kek.y * c2};
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int i = mandel_i<D>(m), j = mandel_j<D>(m);
      const T ki = (T)k[i], kj = (T)k[j], mkij = (T)(-k[i] * k[j]);
      cpx<T> g;
      g.x = fma(mkij, Sk.x, fma(ki, Q[j].x, Q[i].x * kj));
      g.y = fma(mkij, Sk.y, fma(ki, Q[j].y, Q[i].y * kj));
      if (i != j) {
        g.x *= s2;
        g.y *= s2;
      }
      if (MODE == PROJ_GAMMA) {
        o[m] = g;
      } else {
        o[m].x = fma((T)-2, g.x, scale * v[m].x);
        o[m].y = fma((T)-2, g.y, scale * v[m].y);
      }
    }
  }
}

// One CTA per tile of TC columns of all NC components (two-level line index: component a,
// column c), one thread per first-stage butterfly (NC x TC x n / R_0, capped at kColThreads).
// The forward transform loads the tile straight from the spectrum; the projection works in
// shared memory; the last inverse stage stores straight back. D is the spatial dimension,
// NC the field's components (D for vector fields, D (D + 1) / 2 for strains).
template <typename T, int D, int NC, int MODE>
__global__ void __launch_bounds__(kColThreads<T>, 2)
k_proj(cpx<T>* S, AxisPlan P, const cpx<T>* __restrict__ twg, ProjGeom g, int TC,
       int TCp, const Scalars* sc, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  const int n = P.n;
  cpx<T>* sm = smem_c<T>();
  // buffers each hold the NC component tiles (n x TCp, component stride cstr)
  const int cstr = n * TCp;
  const int bufA = n, bufB = n + NC * cstr;
  __shared__ AxisPlan Ps;
  if (threadIdx.x == 0) Ps = P;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = twg[i];
  __syncthreads();
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, g.C - c0);
  const int tcl = __ffs(TC) - 1;
  const Loc<T> gl = gcols<T>(S + c0, (int)g.C, (int)g.cs, tcl, ncols);
  const int nl = NC * TC;
  const int nst = Ps.nst;
  // forward DFT of axis 0: first stage from the spectrum, the rest in shared memory
  stage_any<T>(false, &Ps, 0, gl, sloc2<T>(bufA, 1, TCp, cstr, tcl), nl, true, 0);
  __syncthreads();
  int fwd = bufA, other = bufB;
#pragma unroll 1
  for (int st = 1; st < nst; ++st) {
    stage_any<T>(false, &Ps, st, sloc2<T>(fwd, 1, TCp, cstr, tcl),
                 sloc2<T>(other, 1, TCp, cstr, tcl), nl, true, 0);
    __syncthreads();
    const int t = fwd;
    fwd = other;
    other = t;
  }
  const T scale = (T)g.scale;
  // frequencies of this thread's column (fixed over the rows); columns past a ragged tile's
  // end hold stale values that are transformed but never stored
  const int c = threadIdx.x & (TC - 1);
  int kc1 = 0, kc2 = 0;
  {
    const int cc = (int)(c0 + c);
    if (D == 3) {
      const int i1 = fdiv(cc, g.fdnh);
      kc1 = (i1 <= (g.n1 - 1) / 2) ? i1 : i1 - g.n1;
      kc2 = cc - i1 * g.nh;
    } else {
      kc1 = cc;
    }
  }
  for (int j = threadIdx.x >> tcl; j < n; j += blockDim.x >> tcl) {
    int k[3];
    k[0] = (j <= (n - 1) / 2) ? j : j - n;
    k[1] = kc1;
    k[2] = kc2;
    bool inside = true;
    int kk = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      inside = inside && (abs(k[a]) <= g.hw[a]);
      kk += k[a] * k[a];
    }
    cpx<T> v[NC], o[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) v[a] = sm[fwd + a * cstr + j * TCp + c];
    const T coef = (kk > 0 && inside) ? inv_kk<T>(g, scale, kk) : (T)0;
    proj_point<T, D, NC, MODE>(k, coef, kk, scale, v, o);
#pragma unroll
    for (int a = 0; a < NC; ++a) sm[fwd + a * cstr + j * TCp + c] = o[a];
  }
  __syncthreads();
  // inverse DFT of axis 0: stages in shared memory, the last one into the spectrum
  int a = fwd, b = other;
#pragma unroll 1
  for (int st = 0; st < nst - 1; ++st) {
    stage_any<T>(true, &Ps, st, sloc2<T>(a, 1, TCp, cstr, tcl), sloc2<T>(b, 1, TCp, cstr, tcl),
                 nl, true, 0);
    __syncthreads();
    const int t = a;
    a = b;
    b = t;
  }
  stage_any<T>(true, &Ps, nst - 1, sloc2<T>(a, 1, TCp, cstr, tcl), gl, nl, true, 0);
}

// Projection pass of the 3-D scalar problem (Gamma^ only). Gamma^(k) v = k s(k) with
// s = (k . v) / |k|^2 (eq. (proj)), and k_1, k_2 are constant along axis 0: of the three forward
// axis-0 transforms two remain, of X_0 and of Y = k_1 X_1 + k_2 X_2 (combined on load), and of
// the three inverse ones also two, of k_0 s and of s; the outputs of components 1 and 2 are
// k_1 U and k_2 U with U = F_0^{-1} s. One CTA per tile of TC columns, two lines per column.
__device__ __forceinline__ void column_freqs(const ProjGeom& g, long long cc, int* kc1, int* kc2) {
  const int i1 = fdiv((int)cc, g.fdnh);
  *kc1 = (i1 <= (g.n1 - 1) / 2) ? i1 : i1 - g.n1;
  *kc2 = (int)cc - i1 * g.nh;
}

// Gamma^ (or I - 2 Gamma^ for PROJ_EM) node by node on a spectrum already transformed along all
// axes (the strain projection of elasticity, between the forward and the inverse axis-0 column
// passes): blockIdx.y = row j of axis 0, x over the columns, blockIdx.z = request
template <typename T, int D, int NC, int MODE>
__global__ void __launch_bounds__(kThreads)
k_proj_point(cpx<T>* S, ProjGeom g, int n0, T nodes, const Scalars* sc,
             const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  const long long cc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cc >= g.C) return;
  const int j = blockIdx.y;
  int k[3] = {(j <= (n0 - 1) / 2) ? j : j - n0, 0, 0};
  if (D == 3) {
    column_freqs(g, cc, &k[1], &k[2]);
  } else {
    k[1] = (int)cc;
  }
  bool inside = true;
  int kk = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    inside = inside && (abs(k[a]) <= g.hw[a]);
    kk += k[a] * k[a];
  }
  const T scale = (T)g.scale;
  const T coef = (kk > 0 && inside) ? inv_kk<T>(g, scale, kk) : (T)0;
  cpx<T>* p = S + (long long)j * g.C + cc;
  cpx<T> v[NC], o[NC];
#pragma unroll
  for (int a = 0; a < NC; ++a) v[a] = p[(long long)a * g.cs];
  proj_point<T, D, NC, MODE>(k, coef, kk, scale, v, o, nodes);
#pragma unroll
  for (int a = 0; a < NC; ++a) p[(long long)a * g.cs] = o[a];
}

template <typename T, bool SMALLR = false>
__global__ void __launch_bounds__(kColThreads<T>, SMALLR ? 3 : 2)
k_proj_scalar(cpx<T>* S, AxisPlan P, const cpx<T>* __restrict__ twg, ProjGeom g, int TC,
              int TCp, const Scalars* sc, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  const int n = P.n;
  cpx<T>* sm = smem_c<T>();
  const int cstr = n * TCp;  // line t of column c, row j at buf + t * cstr + j * TCp + c
  const int bufA = n, bufB = n + 2 * cstr;
  __shared__ AxisPlan Ps;
  if (threadIdx.x == 0) Ps = P;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = twg[i];
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, g.C - c0);
  const int tcl = __ffs(TC) - 1;
  const int c = threadIdx.x & (TC - 1);
  const long long es = g.C;
  int kc1, kc2;
  column_freqs(g, c0 + c, &kc1, &kc2);
  // load X_0 and Y = k_1 X_1 + k_2 X_2 (columns past a ragged end are zero)
  for (int j = threadIdx.x >> tcl; j < n; j += blockDim.x >> tcl) {
    cpx<T> x0 = {0, 0}, y = {0, 0};
    if (c < ncols) {
      const cpx<T>* col = S + c0 + c + (long long)j * es;
      const cpx<T> x1 = col[g.cs], x2 = col[2 * g.cs];
      x0 = col[0];
      y.x = (T)kc1 * x1.x + (T)kc2 * x2.x;
      y.y = (T)kc1 * x1.y + (T)kc2 * x2.y;
    }
    sm[bufA + j * TCp + c] = x0;
    sm[bufA + cstr + j * TCp + c] = y;
  }
  __syncthreads();
  const int nl = 2 * TC;
  int a = bufA, b = bufB;
#pragma unroll 1
  for (int st = 0; st < Ps.nst; ++st) {
    stage_any<T, SMALLR>(false, &Ps, st, sloc2<T>(a, 1, TCp, cstr, tcl),
                         sloc2<T>(b, 1, TCp, cstr, tcl), nl, true, 0);
    __syncthreads();
    const int t = a;
    a = b;
    b = t;
  }
  // s = (k_0 v_0 + v_Y) scale / |k|^2 (zero at k = 0 and outside Z_N on a double grid); the
  // lines become k_0 s and s
  const T scale = (T)g.scale;
  for (int j = threadIdx.x >> tcl; j < n; j += blockDim.x >> tcl) {
    const int k0 = (j <= (n - 1) / 2) ? j : j - n;
    const bool inside = abs(k0) <= g.hw[0] && abs(kc1) <= g.hw[1] && abs(kc2) <= g.hw[2];
    const int kk = k0 * k0 + kc1 * kc1 + kc2 * kc2;
    const T coef = (kk > 0 && inside) ? inv_kk<T>(g, scale, kk) : (T)0;
    const cpx<T> v0 = sm[a + j * TCp + c], vy = sm[a + cstr + j * TCp + c];
    cpx<T> sv;
    sv.x = fma((T)k0, v0.x, vy.x) * coef;
    sv.y = fma((T)k0, v0.y, vy.y) * coef;
    sm[a + j * TCp + c] = cpx<T>{(T)k0 * sv.x, (T)k0 * sv.y};
    sm[a + cstr + j * TCp + c] = sv;
  }
  __syncthreads();
#pragma unroll 1
  for (int st = 0; st < Ps.nst; ++st) {
    stage_any<T, SMALLR>(true, &Ps, st, sloc2<T>(a, 1, TCp, cstr, tcl),
                         sloc2<T>(b, 1, TCp, cstr, tcl), nl, true, 0);
    __syncthreads();
    const int t = a;
    a = b;
    b = t;
  }
  // components 0, 1, 2 = F_0^{-1}(k_0 s), k_1 U, k_2 U
  if (c < ncols)
    for (int j = threadIdx.x >> tcl; j < n; j += blockDim.x >> tcl) {
      cpx<T>* col = S + c0 + c + (long long)j * es;
      const cpx<T> t0 = sm[a + j * TCp + c], u = sm[a + cstr + j * TCp + c];
      col[0] = t0;
      col[g.cs] = cpx<T>{(T)kc1 * u.x, (T)kc1 * u.y};
      col[2 * g.cs] = cpx<T>{(T)kc2 * u.x, (T)kc2 * u.y};
    }
}

// Post-operator of the lines l0 .. l0 + LB - 1 after their inverse transform: node j of line
// l0 + ll is the real (ll even) or imaginary (ll odd) part of shared-memory complex line
// res + (a * half + ll / 2) * n; the solver's vector update, batches of K nodes whose operands
// are loaded before any use, and the inner-product partial in dacc (for POST_STORE only when
// `dot` is set: a plain operator application has no partial to form).
template <typename T, int D, int POST, int K = (sizeof(T) == 4 ? 4 : (D > 3 ? 1 : 2)), int NC = 0>
__device__ __forceinline__ void line_post_from_smem(const Fields<T>& f, int res, int n, int half,
                                                    int ncomp, long long l0, int LB,
                                                    long long nlines, FastDiv fdn,
                                                    const MatView<T>& mat, const Scalars* sc,
                                                    const OpArgs& args, int negate,
                                                    DotAcc<T>& dacc, bool dot) {
  cpx<T>* sm = smem_c<T>();
  const double* Es = sc != nullptr ? sc->E : args.E;
  T E[D];
#pragma unroll
  for (int a = 0; a < D; ++a) E[a] = (T)Es[a];
  const T omega = (T)(sc != nullptr ? sc->omega : args.omega);
  const T alpha = sc != nullptr ? (T)sc->alpha : (T)0;
  const T beta = sc != nullptr ? (T)sc->beta : (T)0;
  const int which = sc != nullptr ? sc->which : 0;
  const long long cs = f.cs;
  const T* xc = (POST == POST_RICH) ? f.x + (which ? D * cs : 0) : f.x;
  T* xn = (POST == POST_RICH) ? f.x + (which ? 0 : D * cs) : f.x;
  // NC > 0: the line length as a compile-time constant (specialised kernels); the CTA's lines
  // are contiguous, node idx of the tile is node g0 + idx of the grid
  if (NC > 0) n = NC;
  const long long g0 = l0 * n;
  const int ntile = LB * n;
  const int nvalid = (int)min((long long)ntile, (nlines - l0) * n);
  for (int base = 0; base < ntile; base += K * blockDim.x) {
    T o1[K][D], o2[K][D], o3[K][D], ms[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int idx = base + k * blockDim.x + threadIdx.x;
      const bool ok = idx < nvalid;
      const long long g = g0 + idx;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        o1[k][a] = (ok && (POST == POST_RICH || POST == POST_CHEB || POST == POST_EM ||
                           POST == POST_ADD || POST == POST_CG_FUSED))
                       ? xc[a * cs + g] : (T)0;
        o2[k][a] = (ok && (POST == POST_CG || POST == POST_CHEB || POST == POST_CG_FUSED))
                       ? f.p[a * cs + g] : (T)0;
        o3[k][a] = (ok && (POST == POST_CHEB || POST == POST_CG_FUSED)) ? f.r[a * cs + g] : (T)0;
      }
      ms[k] = (ok && POST == POST_EM) ? mat_fetch<T>(mat, g) : (T)0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int idx = base + k * blockDim.x + threadIdx.x;
      if (idx >= nvalid) continue;
      const int ll = NC > 0 ? idx / NC : fdiv(idx, fdn), j = idx - ll * n;
      const long long g = g0 + idx;
      T y[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (a < ncomp) {
          const cpx<T> z = sm[res + (a * half + (ll >> 1)) * n + j];
          y[a] = (ll & 1) ? z.y : z.x;
        } else {
          y[a] = 0;
        }
      }
      if (POST == POST_STORE) {
        for (int a = 0; a < ncomp; ++a) {
          // the sign flip of `negate` as an integer xor of the sign bit, off the FP pipes
          const T o = flip_sign(y[a], negate ? 0x80000000u : 0u);
          f.out[a * cs + g] = o;
          if (f.r) f.r[a * cs + g] = o;
          if (f.p) f.p[a * cs + g] = o;
          if (dot) dacc.add(y[a], y[a]);
        }
      } else if (POST == POST_RICH) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          xn[a * cs + g] = o1[k][a] - omega * y[a];
          dacc.add(y[a], y[a]);
        }
      } else if (POST == POST_CG) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          f.out[a * cs + g] = y[a];
          dacc.add(y[a], o2[k][a]);
        }
      } else if (POST == POST_CHEB) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const T pv = o2[k][a];
          const T rn = o3[k][a] - alpha * y[a];
          f.r[a * cs + g] = rn;
          f.x[a * cs + g] = o1[k][a] + alpha * pv;
          f.p[a * cs + g] = rn - beta * pv;
          dacc.add(rn, rn);
        }
      } else if (POST == POST_CG_FUSED) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const T rn = o3[k][a] - alpha * y[a];
          f.r[a * cs + g] = rn;
          f.x[a * cs + g] = o1[k][a] + alpha * o2[k][a];
          dacc.add(rn, rn);
        }
      } else if (POST == POST_ADD) {
#pragma unroll
        for (int a = 0; a < D; ++a) f.x[a * cs + g] = o1[k][a] + y[a];
      } else if (POST == POST_EM) {
        T w[D], xv[D];
#pragma unroll
        for (int a = 0; a < D; ++a) w[a] = y[a] + (T)2 * omega * E[a];
        mat_shift_solve_s<T, D>(mat, ms[k], omega, w, xv);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const T dx = xv[a] - o1[k][a];
          f.x[a * cs + g] = xv[a];
          dacc.add(dx, dx);
        }
      }
    }
  }
}

// the stopping quantity of one iteration into the solve's history (if it keeps one)
__device__ __forceinline__ void record_history(Scalars* sc, double v) {
  if (sc->hist != nullptr && sc->nhist < sc->hist_cap) sc->hist[sc->nhist] = v;
  sc->nhist += 1;
}

// The scalar part of the solver step after a post-operator, run by one thread of the last CTA
// with the grid's reduced inner product tot0 over `count` nodes (Algorithms 1-4).
template <int POST>
__device__ __forceinline__ void line_inv_finish(Scalars* sc, double tot0, double count) {
  const double mean = tot0 / count;
  if (POST == POST_STORE) {
    // initial residual r_0 = b (x_0 = 0): ||b|| and (r_0, r_0)
    sc->nb = sqrt(mean);
    sc->rr = mean;
    sc->last_res = sqrt(mean);
  } else if (POST == POST_RICH) {
    const double res = sqrt(mean);  // ||C x_{m-1} - b||
    sc->last_res = res;
    if (sc->stop == 1) record_history(sc, res);
    if (!sc->fixed && sc->stop == 1 && res <= sc->tol * sc->nb) {
      sc->done = 1;
      sc->converged = 1;
      sc->result = sc->which;
      return;
    }
    sc->it += 1;
    sc->which ^= 1;
    sc->result = sc->which;
    const double inc = sc->omega * res;  // ||x_m - x_{m-1}||
    sc->last_inc = inc;
    if (sc->stop == 2) record_history(sc, inc);
    if (sc->fixed) {
      if (sc->it >= sc->maxit) sc->done = 1;
    } else if (sc->stop == 2 && inc <= sc->tol * sc->nE) {
      sc->done = 1;
      sc->converged = 1;
    } else if (sc->it >= sc->maxit) {
      sc->done = 1;
    }
  } else if (POST == POST_CG) {
    sc->pAp = mean;
    sc->alpha = sc->rr / mean;
  } else if (POST == POST_CG_FUSED) {
    // x += alpha p, r -= alpha C p done above; (r, r), the stopping test and beta
    const double res = sqrt(mean);
    sc->last_res = res;
    record_history(sc, res);
    sc->it += 1;
    if (sc->fixed) {
      if (sc->it >= sc->maxit) sc->done = 1;
    } else if (res <= sc->tol * sc->nb) {
      sc->done = 1;
      sc->converged = 1;
    } else if (sc->it >= sc->maxit) {
      sc->done = 1;
    }
    sc->beta = mean / sc->rr;
    sc->rr = mean;
  } else if (POST == POST_CHEB) {
    const double res = sqrt(mean);
    sc->last_res = res;
    record_history(sc, res);
    sc->it += 1;
    if (sc->fixed) {
      if (sc->it >= sc->maxit) sc->done = 1;
    } else if (res <= sc->tol * sc->nb) {
      sc->done = 1;
      sc->converged = 1;
    } else if (sc->it >= sc->maxit) {
      sc->done = 1;
    }
    // coefficients of the next step (Algorithm 3, m > 1)
    const double an = 1.0 / (sc->cheb_d + sc->beta / sc->alpha);
    sc->alpha = an;
    sc->beta = -(sc->cheb_c * an * 0.5) * (sc->cheb_c * an * 0.5);
  } else if (POST == POST_EM) {
    const double inc = sqrt(mean);
    sc->last_inc = inc;
    record_history(sc, inc);
    sc->it += 1;
    if (sc->fixed) {
      if (sc->it >= sc->maxit) sc->done = 1;
    } else if (inc <= sc->tol * sc->nE) {
      sc->done = 1;
      sc->converged = 1;
    } else if (sc->it >= sc->maxit) {
      sc->done = 1;
    }
  }
}


// ---------------------------------------------------------------------------------------
// line_inv: inverse real DFT of the contiguous axis + post-operator
// ---------------------------------------------------------------------------------------
template <typename T, int D, int POST, bool SMALLR = false>
__global__ void __launch_bounds__(kThreads, SMALLR ? 3 : kMinBlocks<T>)
k_line_inv(const cpx<T>* S, Fields<T> f, AxisPlan P, const cpx<T>* __restrict__ twg,
           int ncomp, long long nlines, int LB, LineDiv ld, long long scs, MatView<T> mat,
           Scalars* sc, OpArgs args, double* partials, unsigned* counter, int negate,
           const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  if (reqs != nullptr) {
    const ReqDesc<T>& R = reqs[blockIdx.z];
    f = R.fi;
    S = R.S;
    mat = R.mat;
    sc = R.sc;
    partials = R.partials;
    counter = R.counter;
  }
  if (sc != nullptr && sc->done) return;
  const int n = P.n, nh = (n + 1) / 2;
  const int half = LB / 2;
  const int nlc = ncomp * half;
  cpx<T>* sm = smem_c<T>();
  const int b0 = n, b1 = n + nlc * n;  // b1 holds nlc (n + 1): staged half spectra, ping-pong
  __shared__ AxisPlan Ps;
  if (threadIdx.x == 0) Ps = P;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = twg[i];
  const long long l0 = (long long)blockIdx.x * LB;
  const cpx<T> zero = {0, 0};
  // stage the half spectra of the CTA's lines (contiguous per line) asynchronously
  for (int idx = threadIdx.x; idx < ncomp * LB * nh; idx += blockDim.x) {
    const int al = fdiv(idx, P.fdnh), k = idx - al * nh;
    const int a = fdiv(al, ld.lb), ll = al - a * LB;
    if (l0 + ll < nlines) cp_async_elem<T>(sm + b1 + idx, S + a * scs + (l0 + ll) * nh + k);
    else sm[b1 + idx] = zero;
  }
  cp_async_wait_all();
  __syncthreads();
  // pack two Hermitian half spectra (lines 2 pr, 2 pr + 1) into one complex line
  for (int idx = threadIdx.x; idx < nlc * nh; idx += blockDim.x) {
    const int lc = fdiv(idx, P.fdnh), k = idx - lc * nh;
    const int a = fdiv(lc, ld.half), pr = lc - a * half;
    const cpx<T> A = sm[b1 + (a * LB + 2 * pr) * nh + k];
    const cpx<T> B = sm[b1 + (a * LB + 2 * pr + 1) * nh + k];
    const int line = b0 + lc * n;
    if (k == 0) {
      sm[line].x = A.x;
      sm[line].y = B.x;
    } else {
      sm[line + k].x = A.x - B.y;
      sm[line + k].y = A.y + B.x;
      sm[line + n - k].x = A.x + B.y;
      sm[line + n - k].y = B.x - A.y;
    }
  }
  __syncthreads();
  const int res = reg_lines<T, SMALLR>(b0, b1, &Ps, nlc, n, 1, false, true, 0);

  DotAcc<T> dacc;
  line_post_from_smem<T, D, POST>(f, res, n, half, ncomp, l0, LB, nlines, P.fdn, mat, sc, args,
                                  negate, dacc, partials != nullptr);
  if (partials == nullptr) return;
  double acc[1] = {dacc.value()};
  double tot[1];
  if (!reduce_and_last<1>(acc, partials, counter, tot)) return;
  if (threadIdx.x != 0 || sc == nullptr) return;
  line_inv_finish<POST>(sc, tot[0], (double)(nlines * n));
}

// ---------------------------------------------------------------------------------------
// non-conformity of an iterate (Section 4.4): sqrt of the grid mean of |g - x + e|^2 summed
// over the d components, with g = G x and e = E for the Eyre-Milton iterate (0 for the
// conforming solvers); the last CTA writes it to sc->last_res
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_nonconf(const T* __restrict__ g, const T* __restrict__ x, int d, long long nodes,
          double* partials, unsigned* counter, Scalars* sc) {
  double acc[1] = {0.0};
  const long long len = (long long)d * nodes;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const long long a = i / nodes;
    const double e = sc->E[a];  // the macroscopic field of component a (0 for the conforming)
    const double v = (double)g[i] - (double)x[i] + e;
    acc[0] = fma(v, v, acc[0]);
  }
  double tot[1];
  if (!reduce_and_last<1>(acc, partials, counter, tot)) return;
  if (threadIdx.x == 0) sc->last_res = sqrt(tot[0] / (double)nodes);
}

// ---------------------------------------------------------------------------------------
// energy (A(E + x), E + x) and flux <A(E + x)> (eqs. (GaNi), (ev_bounds))
// ---------------------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(kThreads)
k_energy(const T* __restrict__ x, long long nodes, MatView<T> mat, Scalars* sc, double* partials,
         unsigned* counter) {
  double acc[D + 1];
#pragma unroll
  for (int a = 0; a <= D; ++a) acc[a] = 0.0;
  T E[D];
#pragma unroll
  for (int a = 0; a < D; ++a) E[a] = (T)sc->E[a];
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nodes;
       g += (long long)gridDim.x * blockDim.x) {
    T w[D], v[D];
#pragma unroll
    for (int a = 0; a < D; ++a) w[a] = E[a] + (x ? x[a * nodes + g] : (T)0);
    mat_apply<T, D>(mat, g, w, v);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      acc[0] += (double)v[a] * (double)w[a];
      acc[1 + a] += (double)v[a];
    }
  }
  double tot[D + 1];
  if (!reduce_and_last<D + 1>(acc, partials, counter, tot)) return;
  if (threadIdx.x != 0) return;
  sc->energy = tot[0] / (double)nodes;
#pragma unroll
  for (int a = 0; a < D; ++a) sc->flux[a] = tot[1 + a] / (double)nodes;
}

// ---------------------------------------------------------------------------------------
// small vector kernels
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void k_fill_const(T* x, long long nodes, int d, const Scalars* sc) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nodes * d;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = (T)sc->E[i / nodes];
}

// Iterative refinement, start of an inner solve of C d = r in precision T: r_T = (T) r,
// p_T = r_T, d_T = 0, and (r_T, r_T) in FP64 (the inner ||b|| and (r, r)).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_demote(const double* __restrict__ r64, T* __restrict__ r, T* __restrict__ p, T* __restrict__ x,
         long long len, long long nodes, Scalars* sc, double* partials, unsigned* counter) {
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = (T)r64[i];
    r[i] = v;
    p[i] = v;
    x[i] = (T)0;
    acc[0] += (double)v * (double)v;
  }
  double tot[1];
  if (!reduce_and_last<1>(acc, partials, counter, tot)) return;
  if (threadIdx.x != 0) return;
  const double rr = tot[0] / (double)nodes;
  sc->rr = rr;
  sc->nb = sqrt(rr);
  sc->last_res = sqrt(rr);
  sc->beta = 0.0;
}

// precision conversions of whole fields (FP32 operator applications on FP64 arguments)
template <typename T>
__global__ void k_to_working(const double* __restrict__ src, T* __restrict__ dst, long long len) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}
template <typename T>
__global__ void k_to_double(const T* __restrict__ src, double* __restrict__ dst, long long len) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

// Iterative refinement, end of an inner solve: x_64 += (double) d_T
template <typename T>
__global__ void k_promote(double* __restrict__ x64, const T* __restrict__ dx, long long len) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    x64[i] += (double)dx[i];
}

// half spectrum of grid N (scaled by `scale`) placed into the zeroed half spectrum of grid M
// at the same signed frequencies (prolongation, eq. (ev_bounds)); D = 2 or 3
template <typename T>
__global__ void k_pad_spectrum(const cpx<T>* __restrict__ Sn, cpx<T>* __restrict__ Sm, int D,
                               int n0, int n1, int nh, int m0, int m1, int mh, T scale,
                               long long nlen, long long mlen) {
  const long long per = (long long)n0 * n1 * nh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per * D;
       i += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(i / per);
    long long r = i - a * per;
    const int k2 = (int)(r % nh);
    r /= nh;
    const int j1 = (int)(r % n1);
    const int j0 = (int)(r / n1);
    const int s0 = j0 <= (n0 - 1) / 2 ? j0 : j0 - n0;
    const int s1 = j1 <= (n1 - 1) / 2 ? j1 : j1 - n1;
    const int t0 = s0 >= 0 ? s0 : s0 + m0;
    const int t1 = s1 >= 0 ? s1 : s1 + m1;
    cpx<T> v = Sn[a * nlen + i - a * per];
    v.x *= scale;
    v.y *= scale;
    Sm[a * mlen + ((long long)t0 * m1 + t1) * mh + k2] = v;
  }
}

// half spectrum of grid N taken from the half spectrum of grid M (M >= N per axis) at the same
// signed frequencies, scaled by `scale` (restriction of a trigonometric polynomial of order N,
// the inverse of k_pad_spectrum); D = 2 or 3
template <typename T>
__global__ void k_crop_spectrum(const cpx<T>* __restrict__ Sm, cpx<T>* __restrict__ Sn, int D,
                                int n0, int n1, int nh, int m0, int m1, int mh, T scale,
                                long long nlen, long long mlen) {
  const long long per = (long long)n0 * n1 * nh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per * D;
       i += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(i / per);
    long long r = i - a * per;
    const int k2 = (int)(r % nh);
    r /= nh;
    const int j1 = (int)(r % n1);
    const int j0 = (int)(r / n1);
    const int s0 = j0 <= (n0 - 1) / 2 ? j0 : j0 - n0;
    const int s1 = j1 <= (n1 - 1) / 2 ? j1 : j1 - n1;
    const int t0 = s0 >= 0 ? s0 : s0 + m0;
    const int t1 = s1 >= 0 ? s1 : s1 + m1;
    cpx<T> v = Sm[a * mlen + ((long long)t0 * m1 + t1) * mh + k2];
    v.x *= scale;
    v.y *= scale;
    Sn[a * nlen + i - a * per] = v;
  }
}

template <typename T>
__global__ void k_scale_spectrum(cpx<T>* S, long long len, T scale) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    S[i].x *= scale;
    S[i].y *= scale;
  }
}

}  // namespace hom
