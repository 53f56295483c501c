// Register-resident odd DFTs and the Stockham stage that drives them.
//
// A transform of eq. (DFT) along one axis of odd length n = R_0 R_1 ... R_{S-1} runs as S
// self-sorting (Stockham, decimation-in-time) stages. Stage s with radix R and p = R_0 ... R_{s-1}
// takes, for butterfly i < n/R and k = i mod p,
//   u_r = in[i + r n/R] * w^{r k},  w = exp(-2 pi i / (p R)),   r < R,
//   U = DFT_R(u),   out[(i - k) R + k + r p] = U_r,
// so the output is in natural order after the last stage. Each R_s is an odd number <= 31 and
// DFT_R is computed entirely in registers: a prime R by pairing the terms r and R - r (a cosine
// and a sine part per output pair), a composite R = A B by the same Cooley-Tukey split in
// registers with compile-time indices and constant twiddles. The planner groups the prime
// factors of n into as few such radices as fit in registers, so most axes need two stages.
// The inverse transform (eq. (DFT), no scaling) is conj(F(conj(.))): imaginary parts are
// negated on the load of a transform's first stage and the store of its last (bit 0 / bit 1 of
// a stage's cj flags).
#pragma once
#include <cmath>

#include "common.cuh"

namespace hom {

// ---------------------------------------------------------------------------------------
// constants cos/sin(2 pi j / R) for every odd R <= 31
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int reg_offset(int R) {
  // sum of the odd sizes below R, starting at 3
  return R <= 3 ? 0 : reg_offset(R - 2) + (R - 2);
}
constexpr int kRegMax = 31;
constexpr int kRegTable = reg_offset(kRegMax) + kRegMax;  // 255

static __constant__ double c_rcos_d[kRegTable];
static __constant__ double c_rsin_d[kRegTable];
static __constant__ double c_rtan_d[kRegTable];  // tan(2 pi j / R): never infinite for odd R
static __constant__ float c_rcos_f[kRegTable];
static __constant__ float c_rsin_f[kRegTable];

// Fill this translation unit's copies of the tables (each unit that launches register DFTs
// calls it once per device), from long double cos / sin.
static inline cudaError_t upload_reg_tables() {
  double cd[kRegTable], sd[kRegTable], td[kRegTable];
  float cf[kRegTable], sf[kRegTable];
  const long double twopi = 6.283185307179586476925286766559005768L;
  for (int R = 3; R <= kRegMax; R += 2) {
    const int off = reg_offset(R);
    for (int j = 0; j < R; ++j) {
      const long double t = twopi * (long double)j / (long double)R;
      cd[off + j] = (double)cosl(t);
      sd[off + j] = (double)sinl(t);
      td[off + j] = (double)(sinl(t) / cosl(t));
      cf[off + j] = (float)cosl(t);
      sf[off + j] = (float)sinl(t);
    }
  }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_rcos_d, cd, sizeof(cd))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_rsin_d, sd, sizeof(sd))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_rtan_d, td, sizeof(td))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_rcos_f, cf, sizeof(cf))) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_rsin_f, sf, sizeof(sf));
}

template <typename T> __device__ __forceinline__ T rcos(int j);
template <typename T> __device__ __forceinline__ T rsin(int j);
template <> __device__ __forceinline__ double rcos<double>(int j) { return c_rcos_d[j]; }
template <> __device__ __forceinline__ double rsin<double>(int j) { return c_rsin_d[j]; }
template <> __device__ __forceinline__ float rcos<float>(int j) { return c_rcos_f[j]; }
template <> __device__ __forceinline__ float rsin<float>(int j) { return c_rsin_f[j]; }
template <typename T> __device__ __forceinline__ T rtan(int j);
template <> __device__ __forceinline__ double rtan<double>(int j) { return c_rtan_d[j]; }

__host__ __device__ constexpr int smallest_factor(int R) {
  return R % 3 == 0 ? 3 : R % 5 == 0 ? 5 : R % 7 == 0 ? 7 : R % 11 == 0 ? 11 : R % 13 == 0 ? 13
       : R % 17 == 0 ? 17 : R % 19 == 0 ? 19 : R % 23 == 0 ? 23 : R % 29 == 0 ? 29 : R;
}

// ---------------------------------------------------------------------------------------
// forward DFT of R points held in registers, natural order in and out
// ---------------------------------------------------------------------------------------
template <typename T, int R, int A = smallest_factor(R)>
struct RegDft;

// The outputs of a prime R-point DFT from its pair sums u[r] = x_r + x_{R-r} and differences
// u[R-r] = x_r - x_{R-r} (1 <= r <= (R-1)/2), u[0] = x_0 and y0 = the sum of all x_r
template <typename T, int R>
__device__ __forceinline__ void prime_dft_tail(cpx<T> (&u)[R], cpx<T> y0);

// prime R
template <typename T, int R>
struct RegDft<T, R, R> {
  static __device__ __forceinline__ void run(cpx<T> (&u)[R]) {
    constexpr int H = (R - 1) / 2;
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
    prime_dft_tail<T, R>(u, y0);
  }
};

template <typename T, int R>
__device__ __forceinline__ void prime_dft_tail(cpx<T> (&u)[R], cpx<T> y0) {
  constexpr int H = (R - 1) / 2;
  constexpr int off = reg_offset(R);
  cpx<T> o[R];
  o[0] = y0;
#pragma unroll
  for (int s = 1; s <= H; ++s) {
    cpx<T> C, S;
    C.x = fma(rcos<T>(off + s), u[1].x, u[0].x);
    C.y = fma(rcos<T>(off + s), u[1].y, u[0].y);
    S.x = rsin<T>(off + s) * u[R - 1].x;
    S.y = rsin<T>(off + s) * u[R - 1].y;
#pragma unroll
    for (int r = 2; r <= H; ++r) {
      const int j = (r * s) % R;
      C.x = fma(rcos<T>(off + j), u[r].x, C.x);
      C.y = fma(rcos<T>(off + j), u[r].y, C.y);
      S.x = fma(rsin<T>(off + j), u[R - r].x, S.x);
      S.y = fma(rsin<T>(off + j), u[R - r].y, S.y);
    }
    // y_s = C - i S, y_{R-s} = C + i S
    o[s].x = C.x + S.y;
    o[s].y = C.y - S.x;
    o[R - s].x = C.x - S.y;
    o[R - s].y = C.y + S.x;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) u[r] = o[r];
}

// composite R = A * B: A-point DFTs over the stride-B subsequences, twiddles
// exp(-2 pi i j2 k1 / R), B-point DFTs over j2: X[k1 + A k2]
template <typename T, int R, int A>
struct RegDft {
  static __device__ __forceinline__ void run(cpx<T> (&u)[R]) {
    constexpr int B = R / A;
    constexpr int off = reg_offset(R);
    cpx<T> y[R];  // y[k1 * B + j2]
#pragma unroll
    for (int j2 = 0; j2 < B; ++j2) {
      cpx<T> v[A];
#pragma unroll
      for (int j1 = 0; j1 < A; ++j1) v[j1] = u[j2 + B * j1];
      RegDft<T, A>::run(v);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) {
        const int m = (j2 * k1) % R;
        if (m == 0) {
          y[k1 * B + j2] = v[k1];
        } else {
          const T c = rcos<T>(off + m), s = -rsin<T>(off + m);
          y[k1 * B + j2].x = v[k1].x * c - v[k1].y * s;
          y[k1 * B + j2].y = v[k1].x * s + v[k1].y * c;
        }
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      cpx<T> v[B];
#pragma unroll
      for (int j2 = 0; j2 < B; ++j2) v[j2] = y[k1 * B + j2];
      RegDft<T, B>::run(v);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) u[k1 + A * k2] = v[k2];
    }
  }
};

// ---------------------------------------------------------------------------------------
// FP64 stages with cosine-factored twiddles
//
// FP64 work is bound by the number of FP64 instructions, and a complex product with a twiddle
// costs four of them (two multiplications, two fused multiply-adds). With a twiddle written as
// w = c (1 + i t), c = Re w, t = Im w / Re w (c is never zero for odd lengths), u w = c v with
// v = (u_x - t u_y, u_y + t u_x): two fused multiply-adds, and the real factor c rides along
// into the butterfly's own multiply-adds (the factorisation of twiddles for multiply-add units
// of Linzer and Feig, and of Goedecker for radices 2 to 5). A twiddled 3-point DFT then costs
// 18 instructions instead of 20, a twiddled 9-point one 106 instead of 120, an untwiddled
// 9-point one (its internal twiddles factored the same way) 84 instead of 88, an untwiddled
// 27-point one (3 x 9) 404 instead of 436, and a twiddled prime one (5, 7) two fewer per pair
// of terms r, R - r. The stage twiddle tables of FP64 transforms hold (c, t) instead of
// (Re w, Im w). The helpers are written for either precision; FP32 keeps complex products
// (its passes are not bound by FP32 issue, and the folded forms cost the column passes
// registers and occupancy).
// ---------------------------------------------------------------------------------------

// v = u (1 + i t)
template <typename T>
__device__ __forceinline__ cpx<T> tan_rot(cpx<T> u, T t) {
  cpx<T> v;
  v.x = fma(-t, u.y, u.x);
  v.y = fma(t, u.x, u.y);
  return v;
}

// the 3-point outputs y1 = t - i S d, y2 = t + i S d with S = sin(2 pi / 3)
template <typename T>
__device__ __forceinline__ void dft3_tail(cpx<T> t, cpx<T> d, cpx<T>& y1, cpx<T>& y2) {
  const T S = rsin<T>(reg_offset(3) + 1);
  y1.x = fma(S, d.y, t.x);
  y1.y = fma(-S, d.x, t.y);
  y2.x = fma(-S, d.y, t.x);
  y2.y = fma(S, d.x, t.y);
}

// DFT_3 of (a, c1 v1, c2 v2), in place
template <typename T>
__device__ __forceinline__ void dft3_s2(cpx<T>& a, cpx<T>& v1, cpx<T>& v2, T c1, T c2) {
  const T h = rcos<T>(reg_offset(3) + 1);  // cos(2 pi / 3) = -1/2
  cpx<T> q, s, d, t;
  q.x = c2 * v2.x;
  q.y = c2 * v2.y;
  s.x = fma(c1, v1.x, q.x);
  s.y = fma(c1, v1.y, q.y);
  d.x = fma(c1, v1.x, -q.x);
  d.y = fma(c1, v1.y, -q.y);
  t.x = fma(h, s.x, a.x);
  t.y = fma(h, s.y, a.y);
  a.x += s.x;
  a.y += s.y;
  dft3_tail(t, d, v1, v2);
}

// DFT_3 of (c0 v0, c1 v1, c2 v2), in place; the middle term c0 v0 - s/2 is formed as
// y0 - (3/2) s from y0 = c0 v0 + s
template <typename T>
__device__ __forceinline__ void dft3_s3(cpx<T>& v0, cpx<T>& v1, cpx<T>& v2, T c0, T c1, T c2) {
  cpx<T> q, s, d, t;
  q.x = c2 * v2.x;
  q.y = c2 * v2.y;
  s.x = fma(c1, v1.x, q.x);
  s.y = fma(c1, v1.y, q.y);
  d.x = fma(c1, v1.x, -q.x);
  d.y = fma(c1, v1.y, -q.y);
  v0.x = fma(c0, v0.x, s.x);
  v0.y = fma(c0, v0.y, s.y);
  t.x = fma((T)-1.5, s.x, v0.x);
  t.y = fma((T)-1.5, s.y, v0.y);
  dft3_tail(t, d, v1, v2);
}

// DFT_3 of (a, b, e), in place (the 12-instruction butterfly of RegDft<T, 3>)
template <typename T>
__device__ __forceinline__ void dft3_p(cpx<T>& a, cpx<T>& b, cpx<T>& e) {
  const T h = rcos<T>(reg_offset(3) + 1);
  cpx<T> s, d, t;
  s.x = b.x + e.x;
  s.y = b.y + e.y;
  d.x = b.x - e.x;
  d.y = b.y - e.y;
  t.x = fma(h, s.x, a.x);
  t.y = fma(h, s.y, a.y);
  a.x += s.x;
  a.y += s.y;
  dft3_tail(t, d, b, e);
}

// Second half of the 9-point DFT (3 x 3 split as in RegDft, j = j2 + 3 j1 -> k = k1 + 3 k2):
// u[j2 + 3 k1] holds the output k1 of the 3-point DFT of column j2; the internal twiddles
// exp(-2 pi i j2 k1 / 9) = C_m (1 - i tan(2 pi m / 9)), m = j2 k1, are factored as above.
// Writes X[k1 + 3 k2] to u in natural order.
template <typename T>
__device__ __forceinline__ void dft9_rows(cpx<T> (&u)[9]) {
  constexpr int o9 = reg_offset(9);
  const T C1 = rcos<T>(o9 + 1), C2 = rcos<T>(o9 + 2), C4 = rcos<T>(o9 + 4);
  const T T1 = -rtan<T>(o9 + 1), T2 = -rtan<T>(o9 + 2), T4 = -rtan<T>(o9 + 4);
  // row k1 = 0: (V0[0], V1[0], V2[0]) at u[0], u[1], u[2]
  cpx<T> a0 = u[0], a1 = u[1], a2 = u[2];
  dft3_p(a0, a1, a2);
  // row k1 = 1: (V0[1], V1[1] w^1, V2[1] w^2) at u[3], u[4], u[5]
  cpx<T> b0 = u[3], b1 = tan_rot(u[4], T1), b2 = tan_rot(u[5], T2);
  dft3_s2(b0, b1, b2, C1, C2);
  // row k1 = 2: (V0[2], V1[2] w^2, V2[2] w^4) at u[6], u[7], u[8]
  cpx<T> e0 = u[6], e1 = tan_rot(u[7], T2), e2 = tan_rot(u[8], T4);
  dft3_s2(e0, e1, e2, C2, C4);
  u[0] = a0; u[3] = a1; u[6] = a2;
  u[1] = b0; u[4] = b1; u[7] = b2;
  u[2] = e0; u[5] = e1; u[8] = e2;
}

// the column outputs of the 9-point split, regrouped so that u[j2 + 3 k1] = V_{j2}[k1]
template <typename T>
__device__ __forceinline__ void dft9_regroup(cpx<T> (&u)[9], const cpx<T> (&V)[3][3]) {
#pragma unroll
  for (int j2 = 0; j2 < 3; ++j2)
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) u[3 * k1 + j2] = V[j2][k1];
}

// DFT_9 of u without twiddles on its inputs
template <typename T>
__device__ __forceinline__ void dft9_plain(cpx<T> (&u)[9]) {
  cpx<T> V[3][3];
#pragma unroll
  for (int j2 = 0; j2 < 3; ++j2) {
    V[j2][0] = u[j2];
    V[j2][1] = u[j2 + 3];
    V[j2][2] = u[j2 + 6];
    dft3_p(V[j2][0], V[j2][1], V[j2][2]);
  }
  dft9_regroup(u, V);
  dft9_rows(u);
}

// DFT_9 of (u0, w_1 u1, ..., w_8 u8) with w_r = c_r (1 + i t_r) given as (c_r, t_r) = tw(r);
// each column of the split takes its own three
template <typename T, typename TW>
__device__ __forceinline__ void dft9_tw(cpx<T> (&u)[9], TW tw) {
  cpx<T> V[3][3];
  {
    const cpx<T> w3 = tw(3), w6 = tw(6);
    V[0][0] = u[0];
    V[0][1] = tan_rot(u[3], w3.y);
    V[0][2] = tan_rot(u[6], w6.y);
    dft3_s2(V[0][0], V[0][1], V[0][2], w3.x, w6.x);
  }
#pragma unroll
  for (int j2 = 1; j2 < 3; ++j2) {
    const cpx<T> wa = tw(j2), wb = tw(j2 + 3), wc = tw(j2 + 6);
    V[j2][0] = tan_rot(u[j2], wa.y);
    V[j2][1] = tan_rot(u[j2 + 3], wb.y);
    V[j2][2] = tan_rot(u[j2 + 6], wc.y);
    dft3_s3(V[j2][0], V[j2][1], V[j2][2], wa.x, wb.x, wc.x);
  }
  dft9_regroup(u, V);
  dft9_rows(u);
}

// DFT_27 of u without twiddles on its inputs, split 3 x 9 as in RegDft (j = j2 + 9 j1 ->
// k = k1 + 3 k2): 3-point DFTs over the columns j2, then for each k1 the 9-point DFT over j2 of
// the column outputs times exp(-2 pi i j2 k1 / 27), factored as above
template <typename T>
__device__ __forceinline__ void dft27_plain(cpx<T> (&u)[27]) {
  constexpr int o27 = reg_offset(27);
#pragma unroll
  for (int j2 = 0; j2 < 9; ++j2) dft3_p(u[j2], u[j2 + 9], u[j2 + 18]);
  // the column outputs k1 sit at u[j2 + 9 k1]
  cpx<T> w0[9], w1[9], w2[9];
#pragma unroll
  for (int j2 = 0; j2 < 9; ++j2) {
    w0[j2] = u[j2];
    w1[j2] = u[j2 + 9];
    w2[j2] = u[j2 + 18];
  }
  dft9_plain(w0);
  dft9_tw(w1, [&](int r) { return cpx<T>{rcos<T>(o27 + r), -rtan<T>(o27 + r)}; });
  dft9_tw(w2, [&](int r) { return cpx<T>{rcos<T>(o27 + 2 * r), -rtan<T>(o27 + 2 * r)}; });
#pragma unroll
  for (int k2 = 0; k2 < 9; ++k2) {
    u[3 * k2] = w0[k2];
    u[1 + 3 * k2] = w1[k2];
    u[2 + 3 * k2] = w2[k2];
  }
}

// DFT_R of a prime R with twiddled inputs, (u0, w_1 u1, ..., w_{R-1} u_{R-1}), (c_r, t_r) =
// tw[r * step]: the pair sum and difference of terms r and R - r become c_r v_r + q and
// c_r v_r - q with q = c_{R-r} v_{R-r} (one multiplication and two multiply-adds a part), 12
// instructions a pair instead of 14 with complex twiddle products
template <typename T, int R>
__device__ __forceinline__ void dft_prime_twiddled(cpx<T> (&u)[R], const cpx<T>* tw, int step) {
  constexpr int H = (R - 1) / 2;
  cpx<T> y0 = u[0];
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    const cpx<T> wa = tw[r * step], wb = tw[(R - r) * step];
    const cpx<T> va = tan_rot(u[r], wa.y), vb = tan_rot(u[R - r], wb.y);
    cpx<T> q;
    q.x = wb.x * vb.x;
    q.y = wb.x * vb.y;
    u[r].x = fma(wa.x, va.x, q.x);
    u[r].y = fma(wa.x, va.y, q.y);
    u[R - r].x = fma(wa.x, va.x, -q.x);
    u[R - r].y = fma(wa.x, va.y, -q.y);
    y0.x += u[r].x;
    y0.y += u[r].y;
  }
  prime_dft_tail<T, R>(u, y0);
}

// the untwiddled FP64 9- and 27-point DFTs with factored internal twiddles (in FP32 they cost
// registers in the column passes and gained nothing: its passes are not bound by FP32 issue)
template <>
struct RegDft<double, 9, 3> {
  static __device__ __forceinline__ void run(cpx<double> (&u)[9]) { dft9_plain(u); }
};
template <>
struct RegDft<double, 27, 3> {
  static __device__ __forceinline__ void run(cpx<double> (&u)[27]) { dft27_plain(u); }
};

// u_r *= w_r for r >= 1, w_r = (c_r, t_r) from tw[r * step]: u w = c (u_x - t u_y, u_y + t u_x),
// four instructions, as a complex product
template <typename T, int R>
__device__ __forceinline__ void apply_twiddles(cpx<T> (&u)[R], const cpx<T>* tw, int step) {
#pragma unroll
  for (int r = 1; r < R; ++r) {
    const cpx<T> w = tw[r * step];
    const T ux = u[r].x;
    u[r].x = w.x * fma(-w.y, u[r].y, ux);
    u[r].y = w.x * fma(w.y, ux, u[r].y);
  }
}

// the radices whose twiddled DFT folds the twiddle cosines into its own multiply-adds
template <int R>
__host__ __device__ constexpr bool folds_twiddles() {
  return R == 3 || R == 5 || R == 7 || R == 9;
}

// DFT_R of (u0, w_1 u1, ..., w_{R-1} u_{R-1}) in a twiddled stage, w_r = (c_r, t_r) from
// tw[r * step]
template <typename T, int R>
__device__ __forceinline__ void dft_twiddled(cpx<T> (&u)[R], const cpx<T>* tw, int step) {
  if constexpr (R == 3) {
    const cpx<T> w1 = tw[step], w2 = tw[2 * step];
    u[1] = tan_rot(u[1], w1.y);
    u[2] = tan_rot(u[2], w2.y);
    dft3_s2(u[0], u[1], u[2], w1.x, w2.x);
  } else if constexpr (R == 9) {
    dft9_tw(u, [&](int r) { return tw[r * step]; });
  } else if constexpr (R == 5 || R == 7) {
    dft_prime_twiddled<T, R>(u, tw, step);
  } else {
    apply_twiddles<T, R>(u, tw, step);
    RegDft<T, R>::run(u);
  }
}

// ---------------------------------------------------------------------------------------
// dynamic shared memory of every pass kernel, addressed with 32-bit element offsets
// ---------------------------------------------------------------------------------------
extern __shared__ __align__(16) unsigned char hom_dyn_smem[];

template <typename T>
__device__ __forceinline__ cpx<T>* smem_c() {
  return reinterpret_cast<cpx<T>*>(hom_dyn_smem);
}

__device__ __forceinline__ int fdiv(int x, const FastDiv& f) {
  const unsigned t = __umulhi(f.mul, (unsigned)x);
  return (int)((t + (((unsigned)x - t) >> f.sh1)) >> f.sh2);
}

// One side of a stage: shared memory (g == nullptr; offsets into hom_dyn_smem as cpx<T>) or a
// global tile (element (l, j) at g + l*ls + j*es, offsets below 2^31).
template <typename T>
struct Loc {
  cpx<T>* g;
  int base;
  int ls;
  int es;
  int lo = 0;        // two-level lines: line l = (l_out << nli_log) + l_in sits at
  int nli_log = -1;  // l_in * ls + l_out * lo (nli_log < 0: one level, l * ls)
  int nin = 1 << 30; // global side: lines whose inner index l_in >= nin (the columns past the
                     // end of a ragged tile) are neither loaded nor stored
};

template <typename T>
__device__ __forceinline__ int line_off(const Loc<T>& L, int l) {
  return L.nli_log < 0 ? l * L.ls
                       : (l & ((1 << L.nli_log) - 1)) * L.ls + (l >> L.nli_log) * L.lo;
}

// v with its sign bit xor-ed with m (0 or the sign bit): the conjugations of the inverse
// transform as one integer operation, off the floating-point pipes
__device__ __forceinline__ double flip_sign(double v, unsigned m) {
  return __hiloint2double(__double2hiint(v) ^ (int)m, __double2loint(v));
}
__device__ __forceinline__ float flip_sign(float v, unsigned m) {
  return __int_as_float(__float_as_int(v) ^ (int)m);
}

// One Stockham stage with radix R over nl lines of length n (p = product of earlier radices).
// Work items: (line, butterfly); colmajor puts the line index fastest.
template <typename T, int R, bool INV>
__device__ __forceinline__ void reg_stage(Loc<T> in, Loc<T> out, int n, int p, int nl,
                                         bool colmajor, int tw_base, FastDiv fd_m, FastDiv fd_p,
                                         int cj) {
  const int m = n / R;
  const int total = nl * m;
  const int ts = n / (p * R);
  // column counts are powers of two except in a ragged last tile
  const bool nl_pow2 = (nl & (nl - 1)) == 0;
  const int nl_log = __ffs(nl) - 1;
  cpx<T>* sm = smem_c<T>();
  const int istride = m * in.es;
  const int ostride = p * out.es;
  // lines past the end of a ragged global tile (inner index >= nin) are skipped
  const int gnli = in.g != nullptr ? in.nli_log : out.nli_log;
  const int gnin = in.g != nullptr ? in.nin : (out.g != nullptr ? out.nin : (1 << 30));
  const int gmask = gnli < 0 ? -1 : (1 << gnli) - 1;
  const unsigned m_in = (INV && (cj & 1)) ? 0x80000000u : 0u;
  const unsigned m_out = (INV && (cj & 2)) ? 0x80000000u : 0u;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int l, i;
    if (colmajor) {
      i = nl_pow2 ? (w >> nl_log) : w / nl;
      l = w - i * nl;
    } else {
      l = fdiv(w, fd_m);
      i = w - l * m;
    }
    if ((l & gmask) >= gnin) continue;
    const int k = i - fdiv(i, fd_p) * p;
    cpx<T> u[R];
    const int io = in.base + line_off(in, l) + i * in.es;
    if (in.g != nullptr) {
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = in.g[io + r * istride];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = sm[io + r * istride];
    }
    if (INV) {
#pragma unroll
      for (int r = 0; r < R; ++r) u[r].y = flip_sign(u[r].y, m_in);
    }
    if constexpr (sizeof(T) == 8 && folds_twiddles<R>()) {
      if (p > 1)
        dft_twiddled<T, R>(u, sm + tw_base, k * ts);
      else
        RegDft<T, R>::run(u);
    } else {
      // one copy of the larger DFTs: the twiddles first, then the plain DFT; FP64 twiddles are
      // (c, t), FP32 ones (Re w, Im w)
      if (p > 1) {
        if constexpr (sizeof(T) == 8) {
          apply_twiddles<T, R>(u, sm + tw_base, k * ts);
        } else {
          const int step = k * ts;
#pragma unroll
          for (int r = 1; r < R; ++r) u[r] = cmul(u[r], sm[tw_base + r * step]);
        }
      }
      RegDft<T, R>::run(u);
    }
    if (INV) {
#pragma unroll
      for (int r = 0; r < R; ++r) u[r].y = flip_sign(u[r].y, m_out);
    }
    const int oo = out.base + line_off(out, l) + ((i - k) * R + k) * out.es;
    if (out.g != nullptr) {
#pragma unroll
      for (int r = 0; r < R; ++r) out.g[oo + r * ostride] = u[r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) sm[oo + r * ostride] = u[r];
    }
  }
}

// Dispatch of one stage on the runtime radix. The radices of the common plans (3, 5, 7, 9) are
// expanded in the calling kernel; the others go through one out-of-line copy per
// precision/direction (a call, whose argument passing and register saves cost local-memory
// traffic, but keeps every kernel's code and register budget small).
template <typename T, bool INV>
__device__ __noinline__ void reg_stage_big(int R, Loc<T> in, Loc<T> out, int n, int p, int nl,
                                           bool colmajor, int tw_base, FastDiv fm, FastDiv fp,
                                           int cj) {
  switch (R) {
    case 11: reg_stage<T, 11, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 13: reg_stage<T, 13, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 15: reg_stage<T, 15, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 17: reg_stage<T, 17, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 19: reg_stage<T, 19, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 21: reg_stage<T, 21, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 23: reg_stage<T, 23, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 25: reg_stage<T, 25, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 27: reg_stage<T, 27, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 29: reg_stage<T, 29, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 31: reg_stage<T, 31, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    default: break;
  }
}

// SMALLR: the caller's plan has no radix above 9 (checked on the host before the launch), so
// the kernel carries no out-of-line path at all (no call sites, lighter register allocation)
template <typename T, bool INV, bool SMALLR = false>
__device__ __forceinline__ void reg_stage_any(int R, Loc<T> in, Loc<T> out, int n, int p, int nl,
                                              bool colmajor, int tw_base, FastDiv fm, FastDiv fp,
                                              int cj) {
  switch (R) {
    case 3: reg_stage<T, 3, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 5: reg_stage<T, 5, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 7: reg_stage<T, 7, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    case 9: reg_stage<T, 9, INV>(in, out, n, p, nl, colmajor, tw_base, fm, fp, cj); break;
    default:
      if constexpr (!SMALLR)
        reg_stage_big<T, INV>(R, in, out, n, p, nl, colmajor, tw_base, fm, fp, cj);
      break;
  }
}

// stage st of plan P (an inverse transform is conj(F(conj .)) over the whole sequence of stages
// 0 .. nst - 1: the first stage conjugates what it loads, the last what it stores, the ones
// between neither)
template <typename T, bool SMALLR = false>
__device__ __forceinline__ void stage_any(bool inv, const AxisPlan* P, int st, Loc<T> in,
                                          Loc<T> out, int nl, bool colmajor, int tw_base) {
  const int cj = (st == 0 ? 1 : 0) | (st == P->nst - 1 ? 2 : 0);
  if (inv)
    reg_stage_any<T, true, SMALLR>(P->radix[st], in, out, P->n, P->pprev[st], nl, colmajor,
                                   tw_base, P->fdm[st], P->fdp[st], cj);
  else
    reg_stage_any<T, false, SMALLR>(P->radix[st], in, out, P->n, P->pprev[st], nl, colmajor,
                                    tw_base, P->fdm[st], P->fdp[st], cj);
}

// shared-memory location helpers
template <typename T>
__device__ __forceinline__ Loc<T> sloc(int base, int ls, int es) {
  return Loc<T>{nullptr, base, ls, es, 0, -1};
}
template <typename T>
__device__ __forceinline__ Loc<T> sloc2(int base, int ls, int es, int lo, int nli_log) {
  return Loc<T>{nullptr, base, ls, es, lo, nli_log};
}
// a global tile of columns: column l at g + l, row j at g + j*es (one level), or component
// l_out of a two-level line index at g + l_out*lo; only the first nin columns exist
template <typename T>
__device__ __forceinline__ Loc<T> gcols(cpx<T>* g, int es, int lo, int nli_log, int nin) {
  return Loc<T>{g, 0, 1, es, lo, nli_log, nin};
}

// All stages of one axis on (2^nli_log inner) x (outer) lines of a two-level layout in shared
// memory, ping-ponging between the buffers at a and b; returns the offset holding the result.
// Ends with a __syncthreads().
template <typename T>
__device__ __forceinline__ int reg_lines2(int a, int b, const AxisPlan* P, int nl, int es, int lo,
                                          int nli_log, bool inv, int tw_base) {
  const int nst = P->nst;
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    stage_any<T>(inv, P, st, sloc2<T>(a, 1, es, lo, nli_log), sloc2<T>(b, 1, es, lo, nli_log), nl,
                 true, tw_base);
    __syncthreads();
    const int t = a;
    a = b;
    b = t;
  }
  return a;
}

// All stages of one axis on nl lines in shared memory (element j of line l at a + l*ls + j*es,
// a and b element offsets of the two ping-pong buffers); returns the offset of the buffer that
// holds the natural-order result. Ends with a __syncthreads().
template <typename T, bool SMALLR = false>
__device__ __forceinline__ int reg_lines(int a, int b, const AxisPlan* P, int nl, int ls, int es,
                                         bool colmajor, bool inv, int tw_base) {
  const int nst = P->nst;
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    stage_any<T, SMALLR>(inv, P, st, sloc<T>(a, ls, es), sloc<T>(b, ls, es), nl, colmajor,
                         tw_base);
    __syncthreads();
    const int t = a;
    a = b;
    b = t;
  }
  return a;
}

// Column transform of a global tile in place (gl: nl columns, one- or two-level as in
// gcols). The first stage loads its butterflies straight from the tile, the stages in between
// ping-pong between the shared-memory buffers at a and b (element (l, j) at l_in + l_out*cstr +
// j*TCp), and the last stage stores straight back; a single-stage plan reads and writes the
// tile directly (each butterfly is then a whole column). No barrier after the final stores.
template <typename T, bool SMALLR = false>
__device__ __forceinline__ void reg_columns_global(Loc<T> gl, int a, int b, int TCp, int cstr,
                                                   int nli_log, int nl, const AxisPlan* P,
                                                   bool inv) {
  const int nst = P->nst;
  if (nst == 1) {
    stage_any<T, SMALLR>(inv, P, 0, gl, gl, nl, true, 0);
    return;
  }
  stage_any<T, SMALLR>(inv, P, 0, gl, sloc2<T>(a, 1, TCp, cstr, nli_log), nl, true, 0);
  __syncthreads();
#pragma unroll 1
  for (int st = 1; st < nst - 1; ++st) {
    stage_any<T, SMALLR>(inv, P, st, sloc2<T>(a, 1, TCp, cstr, nli_log),
                         sloc2<T>(b, 1, TCp, cstr, nli_log), nl, true, 0);
    __syncthreads();
    const int t = a;
    a = b;
    b = t;
  }
  stage_any<T, SMALLR>(inv, P, nst - 1, sloc2<T>(a, 1, TCp, cstr, nli_log), gl, nl, true, 0);
}

}  // namespace hom
