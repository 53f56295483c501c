// Column passes specialised at compile time for two-stage plans n = R1 * R2 (FP32).
//
// The generic column kernels take the radices, strides and work split at run time; for the
// axis lengths of the usual grids the whole transform is fixed at compile time instead:
//   stage 1 (radix R1, p = 1): butterfly i < R2 of a column reads rows i + r R2 straight from
//     the spectrum, and writes rows i R1 + r of a shared-memory tile;
//   stage 2 (radix R2, p = R1): butterfly i < R1 reads rows i + r R1 of the tile, applies the
//     twiddles w_n^{r i}, and writes rows i + r R1 (natural order) straight back.
// The inverse transform is conj(F(conj .)): conjugated on the first load and the last store.
// Threads map to (column, butterfly) with the column fastest, so every row segment of a
// warp's global access is contiguous.
#pragma once
#include <type_traits>

#include "passes.cuh"
#include "tma.cuh"

namespace hom {

// the two-stage plans with specialised kernels: (R1, R2), R1 >= R2, as the planner groups
// the prime factors of 243, 405, 81, 135, 45, 161, 63, 189 and 175
#define HOM_PAIR_PLANS(X) \
  X(27, 9)                \
  X(27, 15)               \
  X(27, 3)                \
  X(15, 9)                \
  X(15, 3)                \
  X(23, 7)                \
  X(21, 3)                \
  X(21, 9)                \
  X(25, 7)

// columns per CTA: 16 (128-byte rows) for the strided pass; for the projection pass the
// widest power of two <= 16 with D * TC * R2 <= 256 threads
template <int R2>
__host__ __device__ constexpr int pair_tc_strided() {
  return 16;
}
template <int D, int R2>
__host__ __device__ constexpr int pair_tc_proj() {
  return D * 16 * R2 <= 256 ? 16 : D * 8 * R2 <= 256 ? 8 : D * 4 * R2 <= 256 ? 4 : 2;
}

template <typename T, int R>
__device__ __forceinline__ void conj_all(cpx<T> (&u)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) u[r].y = -u[r].y;
}

// stage 1 of one column: g = the column's first row (row stride es), t = its shared-memory
// column (row stride TCp)
template <typename T, int R1, int R2, bool INV>
__device__ __forceinline__ void pair_stage1_from_global(const cpx<T>* g, long long es, cpx<T>* t,
                                                        int TCp, int i) {
  cpx<T> u[R1];
#pragma unroll
  for (int r = 0; r < R1; ++r) u[r] = g[(long long)(i + r * R2) * es];
  if (INV) conj_all<T, R1>(u);
  RegDft<T, R1>::run(u);
#pragma unroll
  for (int r = 0; r < R1; ++r) t[(i * R1 + r) * TCp] = u[r];
}

// stage 1 of one column held in shared memory (natural order in s, result in t)
template <typename T, int R1, int R2, bool CONJ_IN>
__device__ __forceinline__ void pair_stage1_shared(const cpx<T>* s, cpx<T>* t, int TCp, int i) {
  cpx<T> u[R1];
#pragma unroll
  for (int r = 0; r < R1; ++r) u[r] = s[(i + r * R2) * TCp];
  if (CONJ_IN) conj_all<T, R1>(u);
  RegDft<T, R1>::run(u);
#pragma unroll
  for (int r = 0; r < R1; ++r) t[(i * R1 + r) * TCp] = u[r];
}

// stage 2 of one column into registers: u[r] = X[i + r R1]
template <typename T, int R1, int R2>
__device__ __forceinline__ void pair_stage2_regs(const cpx<T>* t, const cpx<T>* tw, int TCp, int i,
                                                 cpx<T> (&u)[R2]) {
#pragma unroll
  for (int r = 0; r < R2; ++r) u[r] = t[(i + r * R1) * TCp];
#pragma unroll
  for (int r = 1; r < R2; ++r) u[r] = cmul(u[r], tw[r * i]);
  RegDft<T, R2>::run(u);
}

// ---------------------------------------------------------------------------------------
// strided pass along axis 1 (or a plain pass along axis 0): blockIdx.x = column tile,
// blockIdx.y = batch, blockIdx.z = request; TC * R2 threads
// ---------------------------------------------------------------------------------------
template <typename T, int R1, int R2, bool INV>
__global__ void __launch_bounds__(pair_tc_strided<R2>() * R2)
k_pair_strided(cpx<T>* S, const cpx<T>* __restrict__ twg, long long C, long long es,
               long long bs, const Scalars* sc, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, TC = pair_tc_strided<R2>(), TCp = TC + 1, NT = TC * R2;
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* tile = sm + n;
  for (int i = threadIdx.x; i < n; i += NT) tw[i] = twg[i];
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, C - c0);
  cpx<T>* base = S + (long long)blockIdx.y * bs + c0;
  {
    const int c = threadIdx.x % TC, i = threadIdx.x / TC;
    if (c < ncols) pair_stage1_from_global<T, R1, R2, INV>(base + c, es, tile + c, TCp, i);
  }
  __syncthreads();
  for (int w = threadIdx.x; w < TC * R1; w += NT) {
    const int c = w % TC, i = w / TC;
    if (c >= ncols) continue;
    cpx<T> u[R2];
    pair_stage2_regs<T, R1, R2>(tile + c, tw, TCp, i, u);
    if (INV) conj_all<T, R2>(u);
#pragma unroll
    for (int r = 0; r < R2; ++r) base[(long long)(i + r * R1) * es + c] = u[r];
  }
}

// ---------------------------------------------------------------------------------------
// the same pass on tiles staged by the TMA unit (tma.cuh): a persistent CTA walks the tiles
// (column tile fastest, then batch) with two TC x n tile buffers and loads the next tile by one
// box copy while it transforms the current one. Stage 1 runs in place: butterfly i keeps rows
// i + r R2 and leaves its output r in row i + r R2, so stage 2 finds output position
// i2 + r2 R1 of stage 1 (butterfly r2, output i2) in row r2 + i2 R2. Rows are TC = 16
// values (128 bytes) wide, and each half-warp reads one whole row in both stages.
// extra_tx (0 except under hom_debug_tma_stall) is announced on top of each tile's bytes, so
// that no barrier phase completes and every wait runs out.
// ---------------------------------------------------------------------------------------
template <typename T, int R1, int R2>
__host__ __device__ constexpr size_t pair_strided_tma_smem() {
  // alignment slack, two tiles, twiddles, two barriers
  return 128 + sizeof(cpx<T>) * (size_t)R1 * R2 * (2 * pair_tc_strided<R2>() + 1) + 16;
}

template <typename T, int R1, int R2, bool INV>
__global__ void __launch_bounds__(pair_tc_strided<R2>() * R2)
k_pair_strided_tma(const __grid_constant__ CUtensorMap map, cpx<T>* S,
                   const cpx<T>* __restrict__ twg, long long C, long long es, long long bs,
                   int ntc, int ntiles, const Scalars* sc, unsigned* wait_errors,
                   unsigned extra_tx) {
  wait_prior_grid();
  constexpr int n = R1 * R2, TC = pair_tc_strided<R2>(), NT = TC * R2;
  constexpr unsigned kTileBytes = (unsigned)(sizeof(cpx<T>) * TC * n);
  if (sc != nullptr && sc->done) return;
  unsigned char* raw = hom_dyn_smem;
  const unsigned a0 = smem_addr(raw);
  raw += ((a0 + 127u) & ~127u) - a0;
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(raw);  // tile b at buf + b * TC * n
  cpx<T>* tw = buf + 2 * TC * n;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tw + n);
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += NT) tw[i] = twg[i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) {
    mbar_expect_tx(&bar[0], kTileBytes + extra_tx);
    tma_load_3d(buf, &map, (t % ntc) * TC, 0, t / ntc, &bar[0]);
  }
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    const int b = it & 1;
    cpx<T>* tile = buf + b * TC * n;
    const int tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) {
      // the other buffer was last accessed before the fence and barrier that ended the
      // previous tile
      mbar_expect_tx(&bar[b ^ 1], kTileBytes + extra_tx);
      tma_load_3d(buf + (b ^ 1) * TC * n, &map, (tn % ntc) * TC, 0, tn / ntc, &bar[b ^ 1]);
    }
    const bool ok = mbar_wait(&bar[b], (unsigned)(it >> 1) & 1u);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        if (wait_errors != nullptr) atomicAdd(wait_errors, 1u);
        // let the copy in flight into the other buffer land before the CTA's memory goes
        if (tn < ntiles) mbar_wait(&bar[b ^ 1], (unsigned)((it + 1) >> 1) & 1u);
      }
      return;
    }
    const long long c0 = (long long)(t % ntc) * TC;
    const int ncols = (int)min((long long)TC, C - c0);
    {
      const int c = tid % TC, i = tid / TC;
      cpx<T> u[R1];
#pragma unroll
      for (int r = 0; r < R1; ++r) u[r] = tile[(i + r * R2) * TC + c];
      if (INV) conj_all<T, R1>(u);
      RegDft<T, R1>::run(u);
#pragma unroll
      for (int r = 0; r < R1; ++r) tile[(i + r * R2) * TC + c] = u[r];
    }
    __syncthreads();
    cpx<T>* base = S + (long long)(t / ntc) * bs + c0;
    for (int w = tid; w < TC * R1; w += NT) {
      const int c = w % TC, i2 = w / TC;
      if (c >= ncols) continue;
      cpx<T> u[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) u[r] = tile[(r + i2 * R2) * TC + c];
#pragma unroll
      for (int r = 1; r < R2; ++r) u[r] = cmul(u[r], tw[r * i2]);
      RegDft<T, R2>::run(u);
      if (INV) conj_all<T, R2>(u);
#pragma unroll
      for (int r = 0; r < R2; ++r) base[(long long)(i2 + r * R1) * es + c] = u[r];
    }
    // this tile's shared-memory accesses come before the TMA's next write to the buffer
    fence_proxy_async_smem();
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// axis-1 pass of components 1 and 2 in the two-line chain of the 3-D scalar projection
// (blockIdx.x = column tile, blockIdx.y = plane i0, blockIdx.z = request; 2 * TC * R2 threads).
// k_1 is the axis-1 frequency of a row, k_2 = the column index (the half axis).
//   forward: component 1 <- Y = k_1 F_1[X_1] + k_2 F_1[X_2] (only Y reaches the projection)
//   inverse: component 1 <- F_1^{-1}[k_1 U], component 2 <- k_2 F_1^{-1}[U], U read from
//            component 1 (the projection left U = F_0^{-1} s there)
// ---------------------------------------------------------------------------------------
template <typename T, int R1, int R2, bool INV>
__global__ void __launch_bounds__(2 * pair_tc_strided<R2>() * R2)
k_pair_strided2(cpx<T>* S, const cpx<T>* __restrict__ twg, long long C, long long es,
                long long bs, long long cs, const Scalars* sc,
                const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, TC = pair_tc_strided<R2>(), TCp = TC + 1, NT = 2 * TC * R2;
  constexpr int tstr = n * TCp;
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* A = sm + n;  // tile t (0, 1) of column c at A + t * tstr + c (row stride TCp)
  for (int i = threadIdx.x; i < n; i += NT) tw[i] = twg[i];
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, C - c0);
  cpx<T>* base = S + cs + (long long)blockIdx.y * bs + c0;  // component 1, plane i0
  {
    const int c = threadIdx.x % TC, i = (threadIdx.x / TC) % R2, t = threadIdx.x / (TC * R2);
    if (c < ncols) {
      const cpx<T>* src = base + c + (INV ? 0 : t * cs);
      cpx<T> u[R1];
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        u[r] = src[(long long)(i + r * R2) * es];
        if (INV) {
          u[r].y = -u[r].y;
          if (t == 0) {  // k_1 U: the row is the axis-1 frequency
            const int j = i + r * R2;
            const T k1 = (T)(j <= (n - 1) / 2 ? j : j - n);
            u[r].x *= k1;
            u[r].y *= k1;
          }
        }
      }
      RegDft<T, R1>::run(u);
      cpx<T>* dst = A + t * tstr + c;
#pragma unroll
      for (int r = 0; r < R1; ++r) dst[(i * R1 + r) * TCp] = u[r];
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < TC * R1; w += NT) {
    const int c = w % TC, i = w / TC;
    if (c >= ncols) continue;
    cpx<T> u0[R2], u1[R2];
    pair_stage2_regs<T, R1, R2>(A + c, tw, TCp, i, u0);
    pair_stage2_regs<T, R1, R2>(A + tstr + c, tw, TCp, i, u1);
    const T k2 = (T)(c0 + c);
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int j = i + r * R1;
      cpx<T>* e = base + (long long)j * es + c;
      if (!INV) {
        const T k1 = (T)(j <= (n - 1) / 2 ? j : j - n);
        e[0] = cpx<T>{fma(k1, u0[r].x, k2 * u1[r].x), fma(k1, u0[r].y, k2 * u1[r].y)};
      } else {
        e[0] = cpx<T>{u0[r].x, -u0[r].y};
        e[cs] = cpx<T>{k2 * u1[r].x, -k2 * u1[r].y};
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// projection pass: forward DFT of axis 0, Gamma^ (or I - 2 Gamma^), inverse DFT of axis 0, on
// a tile of TC columns of all D components; D * TC * R2 threads. One shared-memory tile per
// component: forward stage 2 and the projection write back the rows they read, and the
// inverse first stage (one butterfly a thread) loads everything before a barrier.
// ---------------------------------------------------------------------------------------
template <typename T, int D, int MODE, int R1, int R2>
__global__ void __launch_bounds__(D * pair_tc_proj<D, R2>() * R2)
k_pair_proj(cpx<T>* S, const cpx<T>* __restrict__ twg, ProjGeom g, const Scalars* sc,
            const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, TC = pair_tc_proj<D, R2>(), TCp = TC + 1, NT = D * TC * R2;
  constexpr int cstr = n * TCp;
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* A = sm + n;  // D tiles, component stride cstr
  for (int i = threadIdx.x; i < n; i += NT) tw[i] = twg[i];
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, g.C - c0);
  const long long es = g.C;
  // this thread's first-stage butterfly (a, i, c), forward and inverse
  const int c1 = threadIdx.x % TC, i1 = (threadIdx.x / TC) % R2, a1 = threadIdx.x / (TC * R2);
  // forward stage 1, from the spectrum
  if (c1 < ncols)
    pair_stage1_from_global<T, R1, R2, false>(S + a1 * g.cs + c0 + c1, es, A + a1 * cstr + c1, TCp,
                                              i1);
  __syncthreads();
  // forward stage 2 of all D components + the projection at the R2 frequencies of item (i, c)
  const T scale = (T)g.scale;
  for (int w = threadIdx.x; w < TC * R1; w += NT) {
    const int c = w % TC, i = w / TC;
    int kc1 = 0, kc2 = 0;
    const int cc = (int)(c0 + c);
    if (D == 3) {
      const int i1c = fdiv(cc, g.fdnh);
      kc1 = (i1c <= (g.n1 - 1) / 2) ? i1c : i1c - g.n1;
      kc2 = cc - i1c * g.nh;
    } else {
      kc1 = cc;
    }
    cpx<T> v[D][R2];
#pragma unroll
    for (int a = 0; a < D; ++a) pair_stage2_regs<T, R1, R2>(A + a * cstr + c, tw, TCp, i, v[a]);
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int j = i + r * R1;
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
      cpx<T> kv = {0, 0};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        kv.x = fma((T)k[a], v[a][r].x, kv.x);
        kv.y = fma((T)k[a], v[a][r].y, kv.y);
      }
      const T coef = (kk > 0 && inside) ? scale / (T)kk : (T)0;
      kv.x *= coef;
      kv.y *= coef;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        cpx<T> o;
        if (MODE == PROJ_GAMMA) {
          o.x = (T)k[a] * kv.x;
          o.y = (T)k[a] * kv.y;
        } else {  // (I - 2 Gamma^) v
          o.x = fma((T)(-2 * k[a]), kv.x, scale * v[a][r].x);
          o.y = fma((T)(-2 * k[a]), kv.y, scale * v[a][r].y);
        }
        A[a * cstr + j * TCp + c] = o;
      }
    }
  }
  __syncthreads();
  // inverse stage 1 (conjugated input) in place: all loads, a barrier, all stores
  {
    const cpx<T>* s = A + a1 * cstr + c1;
    cpx<T> u[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) u[r] = s[(i1 + r * R2) * TCp];
    conj_all<T, R1>(u);
    RegDft<T, R1>::run(u);
    __syncthreads();
    cpx<T>* t = A + a1 * cstr + c1;
#pragma unroll
    for (int r = 0; r < R1; ++r) t[(i1 * R1 + r) * TCp] = u[r];
  }
  __syncthreads();
  // inverse stage 2 into the spectrum (conjugated output): item (a, i, c)
  for (int w = threadIdx.x; w < D * TC * R1; w += NT) {
    const int c = w % TC, i = (w / TC) % R1, a = w / (TC * R1);
    if (c >= ncols) continue;
    cpx<T> u[R2];
    pair_stage2_regs<T, R1, R2>(A + a * cstr + c, tw, TCp, i, u);
    conj_all<T, R2>(u);
    cpx<T>* out = S + a * g.cs + c0 + c;
#pragma unroll
    for (int r = 0; r < R2; ++r) out[(long long)(i + r * R1) * es] = u[r];
  }
}

// ---------------------------------------------------------------------------------------
// projection pass of the 3-D scalar problem (Gamma^ only): two lines a column, X_0 and
// Y = k_1 X_1 + k_2 X_2 forward, k_0 s and s inverse (see k_proj_scalar); 2 * TC * R2 threads
// ---------------------------------------------------------------------------------------
// columns per CTA: the widest power of two <= 32 with 2 * TC * R2 <= 320 threads (128-byte rows
// for 243 = 27 * 9; measured 25 % faster than 64-byte rows there)
template <int R2>
__host__ __device__ constexpr int pair_tc_proj_scalar() {
  return 2 * 32 * R2 <= 320 ? 32 : 2 * 16 * R2 <= 320 ? 16 : 2 * 8 * R2 <= 320 ? 8 : 4;
}

// TWO: the two-line chain (k_pair_strided2 on both sides): line 1 is read as Y from component 1
// and U is written back to component 1 alone
template <typename T, int R1, int R2, bool TWO>
__global__ void __launch_bounds__(2 * pair_tc_proj_scalar<R2>() * R2)
k_pair_proj_scalar(cpx<T>* S, const cpx<T>* __restrict__ twg, ProjGeom g, const Scalars* sc,
                   const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, TC = pair_tc_proj_scalar<R2>(), TCp = TC + 1, NT = 2 * TC * R2;
  constexpr int cstr = n * TCp;
  if (reqs != nullptr) {
    S = reqs[blockIdx.z].S;
    sc = reqs[blockIdx.z].sc;
  }
  if (sc != nullptr && sc->done) return;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* A = sm + n;  // line t of column c at A + t * cstr + c (row stride TCp)
  for (int i = threadIdx.x; i < n; i += NT) tw[i] = twg[i];
  const long long c0 = (long long)blockIdx.x * TC;
  const int ncols = (int)min((long long)TC, g.C - c0);
  const long long es = g.C;
  // this thread's first-stage butterfly (t, i, c), forward and inverse
  const int c1 = threadIdx.x % TC, i1 = (threadIdx.x / TC) % R2, t1 = threadIdx.x / (TC * R2);
  {
    int kc1, kc2;
    column_freqs(g, c0 + c1, &kc1, &kc2);
    cpx<T> u[R1];
    const cpx<T>* col = S + c0 + c1;
    if (c1 < ncols) {
      if (t1 == 0 || TWO) {
        const cpx<T>* src = col + (t1 == 0 ? 0 : g.cs);
#pragma unroll
        for (int r = 0; r < R1; ++r) u[r] = src[(long long)(i1 + r * R2) * es];
      } else {
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          const cpx<T>* e = col + (long long)(i1 + r * R2) * es;
          const cpx<T> x1 = e[g.cs], x2 = e[2 * g.cs];
          u[r].x = (T)kc1 * x1.x + (T)kc2 * x2.x;
          u[r].y = (T)kc1 * x1.y + (T)kc2 * x2.y;
        }
      }
      RegDft<T, R1>::run(u);
      cpx<T>* t = A + t1 * cstr + c1;
#pragma unroll
      for (int r = 0; r < R1; ++r) t[(i1 * R1 + r) * TCp] = u[r];
    }
  }
  __syncthreads();
  // forward stage 2 of both lines, then s at the R2 frequencies of item (i, c), in place
  const T scale = (T)g.scale;
  for (int w = threadIdx.x; w < TC * R1; w += NT) {
    const int c = w % TC, i = w / TC;
    int kc1, kc2;
    column_freqs(g, c0 + c, &kc1, &kc2);
    cpx<T> v0[R2], vy[R2];
    pair_stage2_regs<T, R1, R2>(A + c, tw, TCp, i, v0);
    pair_stage2_regs<T, R1, R2>(A + cstr + c, tw, TCp, i, vy);
    const bool in12 = abs(kc1) <= g.hw[1] && abs(kc2) <= g.hw[2];
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int j = i + r * R1;
      const int k0 = (j <= (n - 1) / 2) ? j : j - n;
      const int kk = k0 * k0 + kc1 * kc1 + kc2 * kc2;
      const T coef = (kk > 0 && in12 && abs(k0) <= g.hw[0]) ? scale / (T)kk : (T)0;
      cpx<T> sv;
      sv.x = fma((T)k0, v0[r].x, vy[r].x) * coef;
      sv.y = fma((T)k0, v0[r].y, vy[r].y) * coef;
      A[j * TCp + c] = cpx<T>{(T)k0 * sv.x, (T)k0 * sv.y};
      A[cstr + j * TCp + c] = sv;
    }
  }
  __syncthreads();
  // inverse stage 1 (conjugated input) in place: all loads, a barrier, all stores
  {
    const cpx<T>* s0 = A + t1 * cstr + c1;
    cpx<T> u[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) u[r] = s0[(i1 + r * R2) * TCp];
    conj_all<T, R1>(u);
    RegDft<T, R1>::run(u);
    __syncthreads();
    cpx<T>* t = A + t1 * cstr + c1;
#pragma unroll
    for (int r = 0; r < R1; ++r) t[(i1 * R1 + r) * TCp] = u[r];
  }
  __syncthreads();
  // inverse stage 2 into the spectrum: line 0 -> component 0, line 1 -> k_1 U, k_2 U
  for (int w = threadIdx.x; w < 2 * TC * R1; w += NT) {
    const int c = w % TC, i = (w / TC) % R1, t = w / (TC * R1);
    if (c >= ncols) continue;
    cpx<T> u[R2];
    pair_stage2_regs<T, R1, R2>(A + t * cstr + c, tw, TCp, i, u);
    cpx<T>* out = S + c0 + c;
    if (t == 0 || TWO) {
      cpx<T>* dst = out + (t == 0 ? 0 : g.cs);
#pragma unroll
      for (int r = 0; r < R2; ++r) dst[(long long)(i + r * R1) * es] = cpx<T>{u[r].x, -u[r].y};
    } else {
      int kc1, kc2;
      column_freqs(g, c0 + c, &kc1, &kc2);
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        cpx<T>* e = out + (long long)(i + r * R1) * es;
        e[g.cs] = cpx<T>{(T)kc1 * u[r].x, -(T)kc1 * u[r].y};
        e[2 * g.cs] = cpx<T>{(T)kc2 * u[r].x, -(T)kc2 * u[r].y};
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// line passes (contiguous axis, D = 3, every component): CTA = LBP line pairs of each
// component, two real lines packed into one complex line (a, q) at n + (a LBP + q) n
// ---------------------------------------------------------------------------------------
// nodes per thread whose pre-operator loads are issued together in the specialised line_fwd
constexpr int kPairPreBatch = 2;

// line pairs per CTA: as many as keep the first-stage butterflies D x LBP x R2 within 224
// threads; the line kernels are compiled for four CTAs per SM (at most 72 registers a thread),
// measured 9 % faster per FP32 CG step at 243^3 than 256 threads and three CTAs
template <int D, int R2>
__host__ __device__ constexpr int pair_lbp() {
  return 224 / (D * R2);
}
template <int D, int R2>
__host__ __device__ constexpr int pair_line_threads() {
  return (D * pair_lbp<D, R2>() * R2 + 31) / 32 * 32;
}

// Shared memory of the specialised line_fwd pass, in floats from the 16-byte aligned base: the
// n twiddles; the D x LBP complex lines, which the pre-operator first fills with the D real
// tiles of LB x n nodes, component a at raw0 + a rstride + s_a where s_a (< 4) is the position
// of the tile's first node within its 16-byte segment of the field, so that aligned 16-byte
// vectors of the field are aligned in shared memory too (the tiles end at most 8 D - 4 floats
// past the complex lines); then a phase table of up to kPairTab entries. The whole stays within
// 48 KiB for the 243-point plans, so that four CTAs fit the SM's 196 KiB shared-memory
// configuration: a larger one leaves the kernels that follow with less L1 (a 228 KiB line_fwd
// was measured to slow the next line_inv pass by a third).
constexpr int kPairTab = 64;
template <int D, int R1, int R2>
struct PairFwdSmem {
  static constexpr int n = R1 * R2, LBP = pair_lbp<D, R2>(), ntile = 2 * LBP * n;
  static constexpr int raw0 = (2 * n + 3) / 4 * 4;
  static constexpr int rstride = (ntile + 3) / 4 * 4 + 4;
  static constexpr int slack = 8 * D - 4;
  static constexpr int tab = (2 * n + D * ntile + slack + 3) / 4 * 4;
  static constexpr int bytes = 4 * (tab + kPairTab);
  static_assert(raw0 + (D - 1) * rstride + 3 + ntile <= 2 * n + D * ntile + slack,
                "raw tiles overrun the line buffer's slack");
};

// v[a] for a runtime index a < D, by selects (no local-memory copy of v)
template <int D>
__device__ __forceinline__ int pick(const int (&v)[D], int a) {
  int r = v[0];
#pragma unroll
  for (int i = 1; i < D; ++i) r = a == i ? v[i] : r;
  return r;
}

// Pre-operator of the specialised line_fwd pass for isotropic phase materials with one-byte
// phase indices and at most kPairTab phases, FP32: v = a(phase) w with w = x (PRE_LINEAR) or
// w = r + beta p (CG, w stored as the new p). Each component's tile is one contiguous run of
// nvalid floats of the field, read (and p written) as aligned 16-byte vectors, its unaligned
// head and tail (at most 3 + 3 nodes) node by node; the four phase indices of a vector come from
// the two aligned words that hold them (the phase array is padded by 16 bytes), the table is
// staged in shared memory. x and p must lie at the same offset within 16 bytes (checked by the
// caller).
template <int D, int PRE, int K>
__device__ __forceinline__ void pair_pre_vec(const Fields<float>& f, const float* xin,
                                             float* smf, const int (&Fo)[D], long long g0,
                                             int nvalid, int ntile, const MatView<float>& mat,
                                             float beta, float* stab, DotAcc<float>* dacc) {
  constexpr bool CG = PRE == PRE_CG || PRE == PRE_CG_DOT;
  const int NT = blockDim.x, t = threadIdx.x;
  for (int i = t; i < kPairTab; i += NT) stab[i] = i < mat.nphase ? mat.table[i] : 0.f;
  // nodes of the last tile beyond the grid transform as zeros
  for (int idx = nvalid + t; idx < ntile; idx += NT) {
#pragma unroll
    for (int a = 0; a < D; ++a) smf[Fo[a] + idx] = 0.f;
  }
  __syncthreads();
  const uint8_t* phg = mat.ph8 + g0;
  const int phs = (int)((uintptr_t)phg & 3);
  const uint32_t* phw = reinterpret_cast<const uint32_t*>(phg - phs);
#pragma unroll 1
  for (int a = 0; a < D; ++a) {
    const float* xa = xin + a * f.cs + g0;
    float* pa = CG ? f.p + a * f.cs + g0 : nullptr;
    float* sa = smf + pick<D>(Fo, a);
    const int h = min(nvalid, (int)((4 - (((uintptr_t)xa >> 2) & 3)) & 3));
    const int nb = (nvalid - h) >> 2;
    for (int c0 = t; c0 < nb; c0 += K * NT) {
      float4 xv[K], pv[K];
      uint32_t lo[K], hi[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = c0 + k * NT;
        if (c < nb) {
          xv[k] = __ldg(reinterpret_cast<const float4*>(xa + h + 4 * c));
          if (CG) pv[k] = *reinterpret_cast<const float4*>(pa + h + 4 * c);
          const int wi = (phs + h + 4 * c) >> 2;
          lo[k] = __ldg(phw + wi);
          hi[k] = __ldg(phw + wi + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = c0 + k * NT;
        if (c >= nb) continue;
        const int idx = h + 4 * c;
        const uint32_t ph4 = __funnelshift_r(lo[k], hi[k], ((phs + idx) & 3) * 8);
        float w[4] = {xv[k].x, xv[k].y, xv[k].z, xv[k].w};
        if (CG) {
          w[0] = fmaf(beta, pv[k].x, w[0]);
          w[1] = fmaf(beta, pv[k].y, w[1]);
          w[2] = fmaf(beta, pv[k].z, w[2]);
          w[3] = fmaf(beta, pv[k].w, w[3]);
          *reinterpret_cast<float4*>(pa + idx) = make_float4(w[0], w[1], w[2], w[3]);
        }
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          v[e] = stab[(ph4 >> (8 * e)) & (kPairTab - 1)] * w[e];
          if (PRE == PRE_CG_DOT) dacc->add(w[e], v[e]);
        }
        *reinterpret_cast<float4*>(sa + idx) = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
    // head [0, h) and tail [h + 4 nb, nvalid), node by node
    const int tail0 = h + 4 * nb, nedge = h + nvalid - tail0;
    if (t < nedge) {
      const int idx = t < h ? t : tail0 + (t - h);
      float w = __ldg(xa + idx);
      if (CG) {
        w = fmaf(beta, pa[idx], w);
        pa[idx] = w;
      }
      const float v = stab[phg[idx] & (kPairTab - 1)] * w;
      if (PRE == PRE_CG_DOT) dacc->add(w, v);
      sa[idx] = v;
    }
  }
}

// pre-operator + forward real DFT of the contiguous axis: the pre-operator fills the real tiles
// in shared memory, stage 1 packs each line pair into one complex line on load and runs in
// place (one butterfly per thread, all loads before a barrier, then all stores), stage 2 in
// place (each butterfly reads and writes the same R2 rows), then the two packed real transforms
// are split and stored as half spectra
template <typename T, int D, int PRE, int R1, int R2>
__global__ void __launch_bounds__(pair_line_threads<D, R2>(), 4)
k_pair_line_fwd(Fields<T> f, cpx<T>* S, const cpx<T>* __restrict__ twg, long long nlines,
                long long scs, MatView<T> mat, Scalars* sc, OpArgs args, FastDiv fdn,
                double* partials, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, nh = (n + 1) / 2, LBP = pair_lbp<D, R2>(), LB = 2 * LBP;
  constexpr int NL = D * LBP, items1 = NL * R2;
  if (reqs != nullptr) {
    const ReqDesc<T>& R = reqs[blockIdx.z];
    f = R.ff;
    S = R.S;
    mat = R.mat;
    sc = R.sc;
    partials = R.partials;
  }
  if (sc != nullptr && sc->done) return;
  using L = PairFwdSmem<D, R1, R2>;
  constexpr bool CG = PRE == PRE_CG || PRE == PRE_CG_DOT;
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* lines = sm + n;
  T* smf = reinterpret_cast<T*>(sm);
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
  const long long l0 = (long long)blockIdx.x * LB;
  const long long g0 = l0 * n;
  const int nvalid = (int)min((long long)L::ntile, (nlines - l0) * n);
  // the operand (as the pre-operator picks it: Richardson's current buffer of a pair)
  const T* xin = (f.x != nullptr && sc != nullptr) ? f.x + (sc->which ? D * f.cs : 0) : f.xin;
  int Fo[D];
#pragma unroll
  for (int a = 0; a < D; ++a)
    Fo[a] = L::raw0 + a * L::rstride + (int)(((uintptr_t)(xin + a * f.cs + g0) >> 2) & 3);
  DotAcc<T> dacc;
  static_assert(std::is_same<T, float>::value, "the specialised line passes are FP32");
  const bool vec = mat.kind == MAT_PHASE_ISO &&
                   mat.ph8 != nullptr && mat.nphase >= 1 && mat.nphase <= kPairTab &&
                   (!CG || ((((uintptr_t)xin ^ (uintptr_t)f.p) & 15) == 0));
  if (vec) {
    pair_pre_vec<D, PRE, kPairPreBatch>(f, xin, smf, Fo, g0, nvalid, L::ntile, mat,
                                        sc != nullptr ? (T)sc->beta : (T)0, smf + L::tab, &dacc);
  } else {
    line_pre_to_smem<T, D, PRE, kPairPreBatch, n, true>(f, n, n, LBP, D, l0, LB, nlines, fdn, mat,
                                                        sc, args, &dacc, Fo);
  }
  __syncthreads();
  {
    const int t = threadIdx.x;
    const bool act = t < items1;
    const int i = t % R2, lc = t / R2, a = lc / LBP, q = lc - a * LBP;
    const T* re = smf + pick<D>(Fo, a) + 2 * q * n + i;  // even line of the pair: real part
    cpx<T>* line = lines + lc * n;
    cpx<T> u[R1];
    if (act) {
#pragma unroll
      for (int r = 0; r < R1; ++r) u[r] = cpx<T>{re[r * R2], re[n + r * R2]};
      RegDft<T, R1>::run(u);
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int r = 0; r < R1; ++r) line[i * R1 + r] = u[r];
    }
  }
  __syncthreads();
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
    cpx<T> A, B;
    A.x = (T)0.5 * (zk.x + zm.x);
    A.y = (T)0.5 * (zk.y - zm.y);
    B.x = (T)0.5 * (zk.y + zm.y);
    B.y = (T)-0.5 * (zk.x - zm.x);
    const long long la = l0 + 2 * q;
    if (la < nlines) S[a * scs + la * nh + k] = A;
    if (la + 1 < nlines) S[a * scs + (la + 1) * nh + k] = B;
  }
  if (PRE == PRE_CG_DOT) line_fwd_partial_cg(dacc, partials);
}

// inverse real DFT of the contiguous axis + post-operator: stage 1 reads the two half spectra
// of each line pair straight from the spectrum and unpacks them on the fly (Hermitian
// symmetry: X_j = conj X_{n-j} above the half), stage 2 runs in place, and the post-operator
// reads the real (even line) and imaginary (odd line) parts
template <typename T, int D, int POST, int R1, int R2>
__global__ void __launch_bounds__(pair_line_threads<D, R2>(), 4)
k_pair_line_inv(const cpx<T>* S, Fields<T> f, const cpx<T>* __restrict__ twg, long long nlines,
                long long scs, MatView<T> mat, Scalars* sc, OpArgs args, double* partials,
                unsigned* counter, int negate, FastDiv fdn, const ReqDesc<T>* __restrict__ reqs) {
  wait_prior_grid();
  constexpr int n = R1 * R2, nh = (n + 1) / 2, LBP = pair_lbp<D, R2>(), LB = 2 * LBP;
  constexpr int NL = D * LBP, items1 = NL * R2;
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
  cpx<T>* sm = smem_c<T>();
  cpx<T>* tw = sm;
  cpx<T>* lines = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
  const long long l0 = (long long)blockIdx.x * LB;
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
      cpx<T> A = okA ? ha[jj] : cpx<T>{0, 0};
      cpx<T> B = okB ? hb[jj] : cpx<T>{0, 0};
      if (up) {
        A.y = -A.y;
        B.y = -B.y;
      }
      // Z = A + i B, conjugated for the inverse transform; Z_0 = (A_0.x, B_0.x)
      if (j == 0) {
        u[r].x = A.x;
        u[r].y = -B.x;
      } else {
        u[r].x = A.x - B.y;
        u[r].y = -(A.y + B.x);
      }
    }
    RegDft<T, R1>::run(u);
    cpx<T>* line = lines + lc * n;
#pragma unroll
    for (int r = 0; r < R1; ++r) line[i * R1 + r] = u[r];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < NL * R1; w += blockDim.x) {
    const int i = w % R1;
    cpx<T>* line = lines + (w / R1) * n;
    cpx<T> u[R2];
    pair_stage2_regs<T, R1, R2>(line, tw, 1, i, u);
#pragma unroll
    for (int r = 0; r < R2; ++r) line[i + r * R1] = cpx<T>{u[r].x, -u[r].y};
  }
  __syncthreads();
  DotAcc<T> dacc;
  // Chebyshev and fused CG read three operands a node: smaller batches keep them within the
  // register budget
  line_post_from_smem<T, D, POST, (D > 3) ? 1 : ((POST == POST_CHEB || POST == POST_CG_FUSED) ? 2 : 4), n>(f, n, n, LBP, D, l0, LB, nlines, fdn,
                                                            mat, sc, args, negate, dacc,
                                                            partials != nullptr);
  if (partials == nullptr) return;
  double acc[1] = {dacc.value()};
  double tot[1];
  if (!reduce_and_last<1>(acc, partials, counter, tot)) return;
  if (threadIdx.x != 0 || sc == nullptr) return;
  line_inv_finish<POST>(sc, tot[0], (double)(nlines * n));
}

}  // namespace hom
