// Conjugate gradients in potential coordinates: the FP32 inner solves of the refinement.
//
// The fields of the method are the gradients x = D u of potentials u (D u = F^{-1}[i k u^] per
// component), and G = D (D*D)^{-1} D* is the orthogonal projection onto them. Algorithm 2 on
// C = G A in the field form is therefore the same iteration, in exact arithmetic, as CG on
// K = D* A D for the potential preconditioned by the Laplacian M = D*D (z = r^ / |k|^2): the
// field iterate is x_m = D u_m, the field residual is D z_m and its squared norm is (r, z),
// b = D z_0, (p, C p) in field form is (D p, A D p). The potential's vectors are one complex
// component on the half spectrum instead of d real components, and the passes of one step
// are the two-line chain of the scalar projection taken in the other order:
//   k_pot_inv  : u += alpha p (the previous step's iterate update, deferred to where p is
//                read anyway), p = z + beta p (the direction update of Algorithm 2), then the
//                inverse axis-0 transforms of k_0 s and s with s = i p (components 0 and 1)
//   strided    : inverse axis 1, two lines -> three components (k_pair_strided + strided2)
//   k_pot_line : inverse axis 2, v = A w and the partial of (w, A w) = (p, K p), forward axis 2
//   (k_cg_alpha: alpha = (r, z) / (p, K p); Chebyshev, Algorithm 3, has its alpha already)
//   strided    : forward axis 1, three components -> X_0 and Y = k_1 X_1 + k_2 X_2
//   k_pot_fwd  : forward axis 0, q = K p = -i (k_0 X_0 + Y) / |N|, r -= alpha q,
//                z = r / |k|^2 and (r, z) (the last CTA: beta, the stopping test)
// After a step the stored u lacks that step's alpha p; the field of the iterate (POT_FIELD)
// adds it as it reads u. Chebyshev (Algorithm 3) runs the same passes with p = z - beta p (the
// beta of the step that formed r) and its own coefficient recurrence in the last CTA of
// k_pot_fwd: on M^{-1} K it is the field-form iteration on G A, whose spectrum on the range of
// G it shares.
// Inner products over the half spectrum count k_2 > 0 twice (Hermitian symmetry of real fields).
// With exact integration (Section 2.3) the solve grid is the double grid and Gamma^ keeps only
// the frequencies of Z_N: the preconditioner is zero outside Z_N, so z, the directions and the
// iterate u stay there, and components of r outside Z_N carry no weight in (r, z).
#pragma once
#include "pair_fft.cuh"

namespace hom {

// 1 / |k|^2 of an integer |k|^2 (0 at k = 0)
__device__ __forceinline__ float pot_inv_kk(int kk) { return kk > 0 ? 1.0f / (float)kk : 0.0f; }

// Tiles of the two axis-0 kernels: TC columns of the half spectrum, all n rows, row-major in
// shared memory with pitch TCp. The vector work (direction update, u and r updates, (r, z)) runs
// element by element over the tile with the threads along the columns of a row, kPotU elements
// a thread in flight; the transforms run on the tile as in k_pair_proj_scalar.
constexpr int kPotU = 4;

// Asks L2 to fetch the 128-byte lines of [p, p + bytes) (PTX prefetch.global.L2), spread over the
// CTA's threads, so that loads issued after the transforms of a tile find them on chip
__device__ __forceinline__ void pot_prefetch_l2(const void* p, long long bytes) {
  const char* b = static_cast<const char*>(p);
  const long long first = reinterpret_cast<unsigned long long>(b) & ~127ull;
  const long long end = reinterpret_cast<unsigned long long>(b) + bytes;
  for (long long a = first + 128ll * threadIdx.x; a < end; a += 128ll * blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// columns per tile of the two axis-0 kernels (2 TC R2 threads a CTA): the forward kernel runs
// narrower tiles and more CTAs a SM (243 points on a GB300: 0.097 ms with 8 columns against
// 0.100 ms with 16)
template <int R2>
__host__ __device__ constexpr int pot_tc_inv() {
  return pair_tc_proj_scalar<R2>();
}
template <int R2>
__host__ __device__ constexpr int pot_tc_fwd() {
  return pair_tc_proj_scalar<R2>() / 2;
}

// k_1^2 + k_2^2 of the tile's columns (-1 for a column outside the support Z_N of exact
// integration, whose frequencies the projection drops) and their Hermitian weights (1 at
// k_2 = 0, else 2; zero past a ragged tile's end)
template <int TC>
__device__ __forceinline__ void pot_tile_cols(const ProjGeom& g, long long c0, int ncols,
                                              int* kk12, float* hw) {
  if (threadIdx.x < TC) {
    int kc1 = 0, kc2 = 0;
    if ((int)threadIdx.x < ncols) column_freqs(g, c0 + threadIdx.x, &kc1, &kc2);
    const bool in12 = abs(kc1) <= g.hw[1] && abs(kc2) <= g.hw[2];
    kk12[threadIdx.x] = in12 ? kc1 * kc1 + kc2 * kc2 : -1;
    hw[threadIdx.x] = (int)threadIdx.x < ncols ? (kc2 == 0 ? 1.0f : 2.0f) : 0.0f;
  }
}

// the preconditioner's 1 / |k|^2 at row frequency k_0 of a column (zero at k = 0 and outside
// the support, so that z and the directions stay in Z_N)
__device__ __forceinline__ float pot_zw(int k0, int kk12c, int hw0) {
  return (kk12c >= 0 && abs(k0) <= hw0) ? pot_inv_kk(k0 * k0 + kk12c) : 0.0f;
}

// axis-0 inverse of the potential step: per column tile, the deferred update u += alpha p and
// the direction update p = z + beta p (z = r / |k|^2; in POT_FIELD mode v = u + alpha p, nothing
// stored), s = i v staged in shared memory, then the inverse axis-0 transforms of k_0 s and s
// into spectrum components 0 and 1; 2 TC R2 threads
template <typename T, int R1, int R2, int MODE>
__global__ void __launch_bounds__(2 * pot_tc_inv<R2>() * R2)
k_pot_inv(cpx<T>* S, const cpx<T>* __restrict__ twg, ProjGeom g, PotVecs<T> V,
          const Scalars* sc, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, TC = pot_tc_inv<R2>(), TCp = TC + 1, NT = 2 * TC * R2;
  constexpr int cstr = n * TCp;
  __shared__ int kk12[TC];
  __shared__ float hwc[TC];
  if (reqs != nullptr) {
    const ReqDesc<T>& R = reqs[blockIdx.z];
    S = R.S;
    sc = R.sc;
    V.u = reinterpret_cast<cpx<T>*>(R.fi.x);
    V.r = reinterpret_cast<cpx<T>*>(R.fi.r);
    V.p = reinterpret_cast<cpx<T>*>(R.fi.p);
  }
  if (MODE == POT_STEP && sc->done) return;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* A = sm + n;
  cpx<T>* stage = A + cstr;  // s = i v of the tile, in the second line's buffer
  for (int i = threadIdx.x; i < n; i += NT) tw[i] = twg[i];
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, g.C - c0);
  const long long es = g.C;
  pot_tile_cols<TC>(g, c0, ncols, kk12, hwc);
  __syncthreads();
  // the previous step's u update, u += alpha_u p, is applied here (and in POT_FIELD mode to
  // the value read), where p is loaded anyway: p is still that step's direction. The new
  // direction is z + beta_p p (Algorithm 2: beta_p = beta; Algorithm 3: -beta of that step).
  const T beta = MODE == POT_STEP ? (T)sc->beta_p : (T)0;
  const T alpha = (T)sc->alpha_u;
  const cpx<T>* __restrict__ rg = V.r;
  cpx<T>* __restrict__ ug = V.u;
  cpx<T>* __restrict__ pg = V.p;
  for (int e0 = threadIdx.x; e0 < n * TC; e0 += kPotU * NT) {
    cpx<T> rr[kPotU], pp[kPotU], uu[kPotU];
#pragma unroll
    for (int q = 0; q < kPotU; ++q) {
      const int e = e0 + q * NT, j = e / TC, c = e % TC;
      rr[q] = pp[q] = uu[q] = cpx<T>{0, 0};
      if (e < n * TC && c < ncols) {
        const long long ge = (long long)j * es + c0 + c;
        uu[q] = ug[ge];
        pp[q] = pg[ge];
        if (MODE == POT_STEP) rr[q] = rg[ge];
      }
    }
#pragma unroll
    for (int q = 0; q < kPotU; ++q) {
      const int e = e0 + q * NT, j = e / TC, c = e % TC;
      if (e >= n * TC) continue;
      const cpx<T> un = {fma(alpha, pp[q].x, uu[q].x), fma(alpha, pp[q].y, uu[q].y)};
      cpx<T> v = un;
      if (MODE == POT_STEP) {
        const int k0 = (j <= (n - 1) / 2) ? j : j - n;
        const T w = (T)pot_zw(k0, kk12[c], g.hw[0]);
        v.x = fma(beta, pp[q].x, rr[q].x * w);
        v.y = fma(beta, pp[q].y, rr[q].y * w);
        if (c < ncols) {
          const long long ge = (long long)j * es + c0 + c;
          pg[ge] = v;
          ug[ge] = un;
        }
      }
      stage[j * TCp + c] = cpx<T>{-v.y, v.x};
    }
  }
  __syncthreads();
  // stage 1 of the inverse transforms: line 0 carries k_0 s, line 1 s (conjugated in and out)
  const int c1 = threadIdx.x % TC, i1 = (threadIdx.x / TC) % R2, t1 = threadIdx.x / (TC * R2);
  {
    cpx<T> u[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int j = i1 + r * R2;
      const int k0 = (j <= (n - 1) / 2) ? j : j - n;
      cpx<T> s = stage[j * TCp + c1];
      if (t1 == 0) {
        s.x *= (T)k0;
        s.y *= (T)k0;
      }
      u[r] = cpx<T>{s.x, -s.y};
    }
    __syncthreads();  // the staged tile is read in full before stage 1 overwrites it
    RegDft<T, R1>::run(u);
    cpx<T>* t = A + t1 * cstr + c1;
#pragma unroll
    for (int r = 0; r < R1; ++r) t[(i1 * R1 + r) * TCp] = u[r];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < 2 * TC * R1; w += NT) {
    const int c = w % TC, i = (w / TC) % R1, t = w / (TC * R1);
    if (c >= ncols) continue;
    cpx<T> u[R2];
    pair_stage2_regs<T, R1, R2>(A + t * cstr + c, tw, TCp, i, u);
    cpx<T>* dst = S + (long long)t * g.cs + c0 + c;
#pragma unroll
    for (int r = 0; r < R2; ++r) dst[(long long)(i + r * R1) * es] = cpx<T>{u[r].x, -u[r].y};
  }
}

// axis-0 forward of the potential step: per column tile, the forward axis-0 transforms of X_0
// (component 0) and Y (component 1), stage 2 in place in the tile, then element by element
// q = -i (k_0 X_0 + Y) / |N| = K p (or D* of the field in POT_INIT mode), r -= alpha q,
// z = r / |k|^2 and the partial of (r, z); the last CTA completes the step (beta and the
// stopping test of Algorithm 2 on sqrt((r, z))). The block is rounded up to whole warps for
// the reduction; the threads past 2 TC R2 take no line in stage 1.
template <int R2>
__host__ __device__ constexpr int pot_fwd_threads() {
  return (2 * pot_tc_fwd<R2>() * R2 + 31) / 32 * 32;
}
template <typename T, int R1, int R2, int MODE>
__global__ void __launch_bounds__(pot_fwd_threads<R2>())
k_pot_fwd(const cpx<T>* S, const cpx<T>* __restrict__ twg, ProjGeom g, PotVecs<T> V,
          Scalars* sc, double* partials, unsigned* counter,
          const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, TC = pot_tc_fwd<R2>(), TCp = TC + 1, NT = 2 * TC * R2;
  constexpr int NTW = pot_fwd_threads<R2>(), cstr = n * TCp;
  __shared__ int kk12[TC];
  __shared__ float hwc[TC];
  if (reqs != nullptr) {
    const ReqDesc<T>& R = reqs[blockIdx.z];
    S = R.S;
    sc = R.sc;
    partials = R.partials;
    counter = R.counter;
    V.u = reinterpret_cast<cpx<T>*>(R.fi.x);
    V.r = reinterpret_cast<cpx<T>*>(R.fi.r);
    V.p = reinterpret_cast<cpx<T>*>(R.fi.p);
  }
  if (MODE == POT_UPDATE && sc->done) return;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* A = sm + n;
  for (int i = threadIdx.x; i < n; i += NTW) tw[i] = twg[i];
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, g.C - c0);
  const long long es = g.C;
  const int c1 = threadIdx.x % TC, i1 = (threadIdx.x / TC) % R2, t1 = threadIdx.x / (TC * R2);
  if (threadIdx.x < NT && c1 < ncols)
    pair_stage1_from_global<T, R1, R2, false>(S + t1 * g.cs + c0 + c1, es, A + t1 * cstr + c1,
                                              TCp, i1);
  pot_tile_cols<TC>(g, c0, ncols, kk12, hwc);
  __syncthreads();
  // stage 2 of both lines in place: item (c, i, t) reads and writes rows i + r R1 of its line
  for (int w = threadIdx.x; w < 2 * TC * R1; w += NTW) {
    const int c = w % TC, i = (w / TC) % R1, t = w / (TC * R1);
    if (c >= ncols) continue;
    cpx<T> v[R2];
    cpx<T>* col = A + t * cstr + c;
    pair_stage2_regs<T, R1, R2>(col, tw, TCp, i, v);
#pragma unroll
    for (int r = 0; r < R2; ++r) col[(i + r * R1) * TCp] = v[r];
  }
  __syncthreads();
  const T alpha = MODE == POT_UPDATE ? (T)sc->alpha : (T)0;
  const T scale = (T)g.scale;
  cpx<T>* __restrict__ ug = V.u;
  cpx<T>* __restrict__ rg = V.r;
  cpx<T>* __restrict__ pg = V.p;
  DotAcc<T> dacc;
  for (int e0 = threadIdx.x; e0 < n * TC; e0 += kPotU * NTW) {
    cpx<T> rr[kPotU];
    if (MODE == POT_UPDATE) {
#pragma unroll
      for (int q = 0; q < kPotU; ++q) {
        const int e = e0 + q * NTW, j = e / TC, c = e % TC;
        rr[q] = cpx<T>{0, 0};
        if (e < n * TC && c < ncols) rr[q] = rg[(long long)j * es + c0 + c];
      }
    }
#pragma unroll
    for (int q = 0; q < kPotU; ++q) {
      const int e = e0 + q * NTW, j = e / TC, c = e % TC;
      if (e >= n * TC || c >= ncols) continue;
      const int k0 = (j <= (n - 1) / 2) ? j : j - n;
      const long long ge = (long long)j * es + c0 + c;
      const cpx<T> x0 = A[j * TCp + c], y = A[cstr + j * TCp + c];
      // q = -i scale (k_0 X_0 + Y)
      const T ax = fma((T)k0, x0.x, y.x) * scale;
      const T ay = fma((T)k0, x0.y, y.y) * scale;
      const cpx<T> kq = {ay, -ax};
      cpx<T> rn;
      if (MODE == POT_INIT) {
        rn = kq;
        ug[ge] = cpx<T>{0, 0};
        pg[ge] = cpx<T>{0, 0};
      } else {
        rn = cpx<T>{fma(-alpha, kq.x, rr[q].x), fma(-alpha, kq.y, rr[q].y)};
      }
      rg[ge] = rn;
      const T wz = (T)pot_zw(k0, kk12[c], g.hw[0]) * (T)hwc[c];
      dacc.add(rn.x * wz, rn.x);
      dacc.add(rn.y * wz, rn.y);
    }
  }
  double acc[1] = {dacc.value()};
  double tot[1];
  if (!reduce_and_last<1, NTW / 32>(acc, partials, counter, tot)) return;
  if (threadIdx.x != 0) return;
  const double rz = tot[0];
  if (MODE == POT_INIT) {
    // r_0 = b, z_0 = M^{-1} r_0: ||b|| = sqrt((r_0, z_0)); u = p = 0, so the first direction
    // is p_1 = z_0 whatever beta is (CG: beta = 0; Chebyshev keeps its initial coefficients)
    sc->nb = sqrt(rz);
    sc->rr = rz;
    sc->last_res = sqrt(rz);
    sc->alpha_u = 0.0;
    sc->beta_p = 0.0;
    return;
  }
  // the step's scalar part: ||r_m|| of the field form is sqrt((r, z))
  const double res = sqrt(rz);
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
  sc->alpha_u = sc->alpha;  // u += alpha p of this step, applied by the next direction update
  if (sc->pot_cheb) {
    // Algorithm 3: p_{m+1} = r_{m+1} - beta_m p_m with this step's beta, then the
    // coefficients of the next step
    sc->beta_p = -sc->beta;
    const double an = 1.0 / (sc->cheb_d + sc->beta / sc->alpha);
    sc->alpha = an;
    sc->beta = -(sc->cheb_c * an * 0.5) * (sc->cheb_c * an * 0.5);
  } else {
    // Algorithm 2: beta = (r_m, z_m) / (r_{m-1}, z_{m-1})
    sc->beta = rz / sc->rr;
    sc->beta_p = sc->beta;
  }
  sc->rr = rz;
}

// The line pass of the potential step (contiguous axis, D = 3): the inverse real DFT of the
// three components (stage 1 reads the half spectra of each line pair and unpacks them, as
// k_pair_line_inv), v = A w node by node in place with the partial of (w, v), then the forward
// real DFT of v (stage 1 on the packed lines in place, stage 2, the split into half spectra,
// as k_pair_line_fwd)
template <typename T, int D, int R1, int R2>
__global__ void __launch_bounds__(pair_line_threads<D, R2>(), 4)
k_pot_line(cpx<T>* S, const cpx<T>* __restrict__ twg, long long nlines, long long scs,
           MatView<T> mat, Scalars* sc, double* partials, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, nh = (n + 1) / 2, LBP = pair_lbp<D, R2>(), LB = 2 * LBP;
  constexpr int NL = D * LBP, items1 = NL * R2;
  if (reqs != nullptr) {
    const ReqDesc<T>& R = reqs[blockIdx.z];
    S = R.S;
    mat = R.mat;
    sc = R.sc;
    partials = R.partials;
  }
  if (sc != nullptr && sc->done) return;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* lines = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
  const long long l0 = (long long)blockIdx.x * LB;
  const long long g0 = l0 * n;
  const int nvalid = (int)min((long long)LB * n, (nlines - l0) * n);
  // the tile's material samples are contiguous (LB whole lines); L2 fetches them while the
  // inverse transforms run
  if (mat.kind == MAT_FIELD)
    pot_prefetch_l2(mat.field + g0, (long long)nvalid * sizeof(T));
  else if (mat.ph8 != nullptr)
    pot_prefetch_l2(mat.ph8 + g0, nvalid);
  else
    pot_prefetch_l2(mat.ph16 + g0, 2ll * nvalid);
  // inverse stage 1: the half spectra of lines (2q, 2q + 1) of component a, unpacked
  if (threadIdx.x < items1) {
    const int t = threadIdx.x;
    const int i = t % R2, lc = t / R2;
    const int a = lc / LBP, q = lc - a * LBP;
    const long long la = l0 + 2 * q;
    const bool okA = la < nlines, okB = la + 1 < nlines;
    const cpx<T>* ha = S + a * scs + la * nh;
    const cpx<T>* hb = ha + nh;
    cpx<T> u[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int j = i + r * R2;
      const bool up = j > (n - 1) / 2;
      const int jj = up ? n - j : j;
      cpx<T> Av = okA ? ha[jj] : cpx<T>{0, 0};
      cpx<T> Bv = okB ? hb[jj] : cpx<T>{0, 0};
      if (up) {
        Av.y = -Av.y;
        Bv.y = -Bv.y;
      }
      if (j == 0) {
        u[r].x = Av.x;
        u[r].y = -Bv.x;
      } else {
        u[r].x = Av.x - Bv.y;
        u[r].y = -(Av.y + Bv.x);
      }
    }
    RegDft<T, R1>::run(u);
    cpx<T>* line = lines + lc * n;
#pragma unroll
    for (int r = 0; r < R1; ++r) line[i * R1 + r] = u[r];
  }
  __syncthreads();
  DotAcc<T> dacc;
  if constexpr (R2 <= 9) {
    // inverse stage 2 of the three components of a line pair, and on the nodes it produces
    // v = A w with the partial of (w, v): item (q, i) owns rows i + r R1 of the packed lines
    // (a, q) of every component (real part: line 2q, imaginary part: line 2q + 1) and writes v
    // back where it read; nodes past the grid's end hold zeros and stay zero
    for (int w = threadIdx.x; w < LBP * R1; w += blockDim.x) {
      const int i = w % R1, q = w / R1;
      cpx<T> u[D][R2];
#pragma unroll
      for (int a = 0; a < D; ++a)
        pair_stage2_regs<T, R1, R2>(lines + (a * LBP + q) * n, tw, 1, i, u[a]);
#pragma unroll
      for (int r = 0; r < R2; ++r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int idx = (2 * q + h) * n + i + r * R1;
          T wv[D], v[D];
#pragma unroll
          for (int a = 0; a < D; ++a) wv[a] = h ? -u[a][r].y : u[a][r].x;  // conjugated output
          if (idx < nvalid) {
            mat_eval<T, D>(mat, mat_fetch<T>(mat, g0 + idx), wv, v);
#pragma unroll
            for (int a = 0; a < D; ++a) dacc.add(wv[a], v[a]);
          } else {
#pragma unroll
            for (int a = 0; a < D; ++a) v[a] = (T)0;
          }
#pragma unroll
          for (int a = 0; a < D; ++a) {
            if (h) u[a][r].y = v[a];
            else u[a][r].x = v[a];
          }
        }
      }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        cpx<T>* line = lines + (a * LBP + q) * n;
#pragma unroll
        for (int r = 0; r < R2; ++r) line[i + r * R1] = u[a][r];
      }
    }
    __syncthreads();
  } else {
    // wider second stages (R2 > 9) hold too many registers for the fused form: stage 2 of
    // every line, then the material product node by node
    for (int w = threadIdx.x; w < NL * R1; w += blockDim.x) {
      const int i = w % R1;
      cpx<T>* line = lines + (w / R1) * n;
      cpx<T> u[R2];
      pair_stage2_regs<T, R1, R2>(line, tw, 1, i, u);
#pragma unroll
      for (int r = 0; r < R2; ++r) line[i + r * R1] = cpx<T>{u[r].x, -u[r].y};
    }
    __syncthreads();
    constexpr int KM = 4;  // material samples a thread has in flight
    for (int base = threadIdx.x; base < LB * n; base += KM * blockDim.x) {
      T smp[KM];
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        const int idx = base + k * blockDim.x;
        smp[k] = idx < nvalid ? mat_fetch<T>(mat, g0 + idx) : (T)0;
      }
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        const int idx = base + k * blockDim.x;
        if (idx >= nvalid) continue;
        const int ll = idx / n, j = idx - ll * n, q = ll >> 1, odd = ll & 1;
        T w[D], v[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const cpx<T> z = lines[(a * LBP + q) * n + j];
          w[a] = odd ? z.y : z.x;
        }
        mat_eval<T, D>(mat, smp[k], w, v);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          dacc.add(w[a], v[a]);
          cpx<T>& z = lines[(a * LBP + q) * n + j];
          if (odd) z.y = v[a];
          else z.x = v[a];
        }
      }
    }
    __syncthreads();
  }
  // forward stage 1 on the packed lines, in place: all loads, a barrier, all stores
  {
    const int t = threadIdx.x;
    const bool act = t < items1;
    const int i = t % R2, lc = t / R2;
    cpx<T>* line = lines + lc * n;
    cpx<T> u[R1];
    if (act) {
#pragma unroll
      for (int r = 0; r < R1; ++r) u[r] = line[i + r * R2];
      RegDft<T, R1>::run(u);
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int r = 0; r < R1; ++r) line[i * R1 + r] = u[r];
    }
  }
  __syncthreads();
  // (the 21 x 9 plan of 189 points spills registers in the fused form)
  if constexpr (R2 <= 9 && !(R1 == 21 && R2 == 9)) {
    // forward stage 2 and the split into half spectra together: item (lc, i) runs stage 2 for
    // the rows of residue i and of its mirror R1 - i (mod R1), which between them hold Z[k] and
    // Z[n - k] for every output k of either residue: n - (i + R1 r) = (R1 - i) + R1 (R2 - 1 - r)
    constexpr int R1h = (R1 + 1) / 2;
    for (int w = threadIdx.x; w < NL * R1h; w += blockDim.x) {
      const int i = w % R1h, lc = w / R1h;
      const int a = lc / LBP, q = lc - a * LBP;
      const cpx<T>* line = lines + lc * n;
      cpx<T> u[R2], v[R2];
      pair_stage2_regs<T, R1, R2>(line, tw, 1, i, u);
      if (i > 0) {
        pair_stage2_regs<T, R1, R2>(line, tw, 1, R1 - i, v);
      } else {
#pragma unroll
        for (int r = 0; r < R2; ++r) v[r] = cpx<T>{0, 0};
      }
      const long long la = l0 + 2 * q;
      const bool okA = la < nlines, okB = la + 1 < nlines;
      cpx<T>* outA = S + a * scs + la * nh;
      cpx<T>* outB = outA + nh;
#pragma unroll
      for (int r = 0; r < R2; ++r) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          if (m == 1 && i == 0) continue;
          const int k = m == 0 ? i + r * R1 : (R1 - i) + r * R1;
          if (k >= nh) continue;
          // Z[k] and Z[n - k]; residue 0 is its own mirror (Z[n - R1 r] = Z[R1 (R2 - r)])
          const cpx<T> zk = m == 0 ? u[r] : v[r];
          const cpx<T> zm = m == 1 ? u[R2 - 1 - r] : (i == 0 ? u[(R2 - r) % R2] : v[R2 - 1 - r]);
          cpx<T> Ah, Bh;
          Ah.x = (T)0.5 * (zk.x + zm.x);
          Ah.y = (T)0.5 * (zk.y - zm.y);
          Bh.x = (T)0.5 * (zk.y + zm.y);
          Bh.y = (T)-0.5 * (zk.x - zm.x);
          if (okA) outA[k] = Ah;
          if (okB) outB[k] = Bh;
        }
      }
    }
  } else {
    for (int w = threadIdx.x; w < NL * R1; w += blockDim.x) {
      const int i = w % R1;
      cpx<T>* line = lines + (w / R1) * n;
      cpx<T> u[R2];
      pair_stage2_regs<T, R1, R2>(line, tw, 1, i, u);
#pragma unroll
      for (int r = 0; r < R2; ++r) line[i + r * R1] = u[r];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NL * nh; idx += blockDim.x) {
      const int lc = idx / nh, k = idx - lc * nh;
      const int a = lc / LBP, q = lc - a * LBP;
      const cpx<T> zk = lines[lc * n + k];
      const cpx<T> zm = lines[lc * n + (k ? n - k : 0)];
      cpx<T> Ah, Bh;
      Ah.x = (T)0.5 * (zk.x + zm.x);
      Ah.y = (T)0.5 * (zk.y - zm.y);
      Bh.x = (T)0.5 * (zk.y + zm.y);
      Bh.y = (T)-0.5 * (zk.x - zm.x);
      const long long la = l0 + 2 * q;
      if (la < nlines) S[a * scs + la * nh + k] = Ah;
      if (la + 1 < nlines) S[a * scs + (la + 1) * nh + k] = Bh;
    }
  }
  line_fwd_partial_cg(dacc, partials);
}

}  // namespace hom
