// Odd mixed-radix FFT engine working on lines held in shared memory.
//
// Transform of eq. (DFT) along one axis of odd length n = prod R_s, every R_s an odd prime
// <= 31. Each stage is one self-sorting (Stockham, decimation in time) radix-R step: for the
// butterfly i of a line, with p = product of the radices already done and k = i mod p,
//   u_r = src[i + r n/R] * w^{r k}, w = exp(-2 pi i / (p R)),
//   U = DFT_R(u),  dst[(i - k) R + k + r p] = U_r,
// so the output comes out in natural order after the last stage. Each output pair (s, R - s)
// of the radix-R DFT costs (R-1)/2 real-by-complex products for its cosine part and as many
// for its sine part. The inverse transform (no scaling, eq. (DFT)) is conj(F(conj(.))),
// applied by negating imaginary parts at every load and store of a stage.
#pragma once
#include "common.cuh"

namespace hom {

// cos / sin (2 pi j / R) for the supported radices, filled by upload_dft_constants().
constexpr int kRadices[] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};
constexpr int kNumRadices = 10;
__host__ __device__ constexpr int radix_offset(int R) {
  return R == 3 ? 0 : R == 5 ? 3 : R == 7 ? 8 : R == 11 ? 15 : R == 13 ? 26 : R == 17 ? 39
       : R == 19 ? 56 : R == 23 ? 75 : R == 29 ? 98 : R == 31 ? 127 : -1;
}
constexpr int kDftTable = 158;

static __constant__ double c_cos_d[kDftTable];
static __constant__ double c_sin_d[kDftTable];
static __constant__ float c_cos_f[kDftTable];
static __constant__ float c_sin_f[kDftTable];

template <typename T> __device__ __forceinline__ T dcos(int j);
template <typename T> __device__ __forceinline__ T dsin(int j);
template <> __device__ __forceinline__ double dcos<double>(int j) { return c_cos_d[j]; }
template <> __device__ __forceinline__ double dsin<double>(int j) { return c_sin_d[j]; }
template <> __device__ __forceinline__ float dcos<float>(int j) { return c_cos_f[j]; }
template <> __device__ __forceinline__ float dsin<float>(int j) { return c_sin_f[j]; }

// One Stockham stage over nl lines: element j of line l sits at l*ls + j*es.
// colmajor selects the work-item order (line index fastest when lines are adjacent columns).
// The radix-R DFT u_s <- sum_r u_r exp(-2 pi i r s / R) is formed from the pairs
// a_r = u_r + u_{R-r} (kept in u[r]) and b_r = u_r - u_{R-r} (kept in u[R-r]); each output
// pair (s, R-s) is written to shared memory as soon as it is complete.
template <typename T, int R, bool INV>
__device__ __forceinline__ void fft_stage(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst,
                                          int n, int p, int nl, int ls, int es, bool colmajor,
                                          const cpx<T>* __restrict__ tw) {
  constexpr int H = (R - 1) / 2;
  constexpr int off = radix_offset(R);
  const int m = n / R;
  const int total = nl * m;
  const int ts = n / (p * R);  // twiddle stride in the length-n table
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int l, i;
    if (colmajor) {
      i = w / nl;
      l = w - i * nl;
    } else {
      l = w / m;
      i = w - l * m;
    }
    const cpx<T>* sp = src + l * ls + i * es;
    cpx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      u[r] = sp[r * m * es];
      if (INV) u[r].y = -u[r].y;
    }
    const int k = i % p;
    if (p > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tw[r * k * ts]);
    }
    cpx<T> y0 = u[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const cpx<T> t = u[r];
      u[r].x = t.x + u[R - r].x;
      u[r].y = t.y + u[R - r].y;
      u[R - r].x = t.x - u[R - r].x;
      u[R - r].y = t.y - u[R - r].y;
      y0.x += u[r].x;
      y0.y += u[r].y;
    }
    cpx<T>* dp = dst + l * ls + ((i - k) * R + k) * es;
    const int os = p * es;
    if (INV) y0.y = -y0.y;
    dp[0] = y0;
#pragma unroll
    for (int s = 1; s <= H; ++s) {
      cpx<T> C, S;
      C.x = fma(dcos<T>(off + s), u[1].x, u[0].x);
      C.y = fma(dcos<T>(off + s), u[1].y, u[0].y);
      S.x = dsin<T>(off + s) * u[R - 1].x;
      S.y = dsin<T>(off + s) * u[R - 1].y;
#pragma unroll
      for (int r = 2; r <= H; ++r) {
        const int j = (r * s) % R;
        C.x = fma(dcos<T>(off + j), u[r].x, C.x);
        C.y = fma(dcos<T>(off + j), u[r].y, C.y);
        S.x = fma(dsin<T>(off + j), u[R - r].x, S.x);
        S.y = fma(dsin<T>(off + j), u[R - r].y, S.y);
      }
      // y_s = C - i S, y_{R-s} = C + i S (then conjugated back for the inverse)
      cpx<T> o1, o2;
      o1.x = C.x + S.y;
      o1.y = INV ? S.x - C.y : C.y - S.x;
      o2.x = C.x - S.y;
      o2.y = INV ? -(C.y + S.x) : C.y + S.x;
      dp[s * os] = o1;
      dp[(R - s) * os] = o2;
    }
  }
}

// Full transform of nl lines, ping-ponging between a and b; returns the buffer holding the
// result. tw[j] = exp(-2 pi i j / n); P points to a copy of the axis plan in shared memory.
// Ends with a __syncthreads(). Not inlined: one copy per precision serves every kernel.
template <typename T, bool INV>
__device__ __noinline__ cpx<T>* fft_lines_dir(cpx<T>* a, cpx<T>* b, const AxisPlan* P, int nl,
                                              int ls, int es, bool colmajor, const cpx<T>* tw) {
  const int nst = P->nst, n = P->n;
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    const int R = P->radix[st];
    const int p = P->pprev[st];
    switch (R) {
      case 3: fft_stage<T, 3, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 5: fft_stage<T, 5, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 7: fft_stage<T, 7, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 11: fft_stage<T, 11, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 13: fft_stage<T, 13, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 17: fft_stage<T, 17, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 19: fft_stage<T, 19, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 23: fft_stage<T, 23, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 29: fft_stage<T, 29, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      case 31: fft_stage<T, 31, INV>(a, b, n, p, nl, ls, es, colmajor, tw); break;
      default: break;
    }
    __syncthreads();
    cpx<T>* t = a;
    a = b;
    b = t;
  }
  return a;
}

template <typename T>
__device__ __forceinline__ cpx<T>* fft_lines(cpx<T>* a, cpx<T>* b, const AxisPlan* P, int nl,
                                             int ls, int es, bool colmajor, bool inv,
                                             const cpx<T>* tw) {
  return inv ? fft_lines_dir<T, true>(a, b, P, nl, ls, es, colmajor, tw)
             : fft_lines_dir<T, false>(a, b, P, nl, ls, es, colmajor, tw);
}

}  // namespace hom
