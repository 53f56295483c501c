// C ABI of libhom (include/hom.h): problem set-up, operator applications and the solver
// drivers of Algorithms 1-4 on top of the fused FFT passes (passes.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/hom.h"
#include "problem.h"

using namespace hom;

namespace hom {
long long& launch_counter() {
  static long long c = 0;
  return c;
}
// per-pass event timing: pairs of events recorded around each launch while enabled
namespace {
struct ProfState {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  cudaEvent_t open[KIND_COUNT] = {};
  size_t used = 0;
  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
};
ProfState& prof_state() {
  static ProfState s;
  return s;
}
}  // namespace
bool profiling() { return prof_state().on; }
void prof_mark(int kind, cudaStream_t st, bool start) {
  ProfState& ps = prof_state();
  cudaEvent_t e = ps.take();
  cudaEventRecord(e, st);
  if (start) {
    ps.open[kind] = e;
  } else {
    ps.marks.push_back({kind, {ps.open[kind], e}});
  }
}
int dynamic_smem_cap() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return optin - 1024;
}
}  // namespace hom

namespace hom {
namespace detail {

cudaError_t& last_cuda_error() {
  static cudaError_t e = cudaSuccess;
  return e;
}

bool spd_eigs(const double* t, int d, double* lo, double* hi) {
  // symmetric check + eigenvalue bounds via Jacobi sweeps on a copy (d <= kMaxComp)
  if (d < 1 || d > kMaxComp) return false;
  double a[kMaxComp][kMaxComp];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) a[i][j] = t[i * d + j];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(a[i][j] - a[j][i]) > 1e-12 * (std::fabs(a[i][j]) + std::fabs(a[j][i]) + 1e-300))
        return false;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        if (i != j) off += a[i][j] * a[i][j];
    if (off < 1e-30) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        if (std::fabs(a[p][q]) < 1e-300) continue;
        const double th = 0.5 * std::atan2(2 * a[p][q], a[q][q] - a[p][p]);
        const double c = std::cos(th), s = std::sin(th);
        for (int k = 0; k < d; ++k) {
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < d; ++k) {
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
      }
  }
  double mn = a[0][0], mx = a[0][0];
  for (int i = 1; i < d; ++i) {
    mn = std::min(mn, a[i][i]);
    mx = std::max(mx, a[i][i]);
  }
  *lo = mn;
  *hi = mx;
  return mn > 0;
}

// (C_p + omega I)^{-1} of every phase of a stiffness table (n x n Mandel matrices, SPD, so
// Gauss-Jordan without pivoting is stable), uploaded for the Eyre-Milton post-operator
int shifted_inverse_table(hom_problem* P, double omega) {
  const int n = P->nc;
  const size_t cnt = (size_t)P->nphase * n * n;
  if (P->d_inv && P->inv_omega == omega) return HOM_OK;
  std::vector<double> tab(cnt), inv(cnt);
  HOM_CUDA(cudaMemcpy(tab.data(), P->d_table, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
  for (int p = 0; p < P->nphase; ++p) {
    double m[kMaxComp][2 * kMaxComp];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        m[i][j] = tab[(size_t)p * n * n + i * n + j] + (i == j ? omega : 0.0);
        m[i][n + j] = i == j ? 1.0 : 0.0;
      }
    for (int c = 0; c < n; ++c) {
      const double piv = m[c][c];
      for (int j = 0; j < 2 * n; ++j) m[c][j] /= piv;
      for (int r = 0; r < n; ++r)
        if (r != c) {
          const double f = m[r][c];
          for (int j = 0; j < 2 * n; ++j) m[r][j] -= f * m[c][j];
        }
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) inv[(size_t)p * n * n + i * n + j] = m[i][n + j];
  }
  if (!P->d_inv) {
    int rc = alloc((void**)&P->d_inv, sizeof(double) * cnt);
    if (rc) return rc;
  }
  HOM_CUDA(cudaMemcpy(P->d_inv, inv.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice));
  P->inv_omega = omega;
  P->e64.mat.inv = P->d_inv;
  return HOM_OK;
}

// allocation-failure injection (hom_debug_fail_alloc): allocations still to pass before one
// fails, or -1 when disarmed
std::atomic<long long>& fail_countdown() {
  static std::atomic<long long> c{-1};
  return c;
}

int alloc(void** p, size_t bytes) {
  long long c = fail_countdown().load();
  while (c >= 0 && !fail_countdown().compare_exchange_weak(c, c - 1)) {
  }
  if (c == 0) {  // the injected failure: the allocation cudaMalloc would refuse on a full device
    *p = nullptr;
    return HOM_ERR_OOM;
  }
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return HOM_ERR_OOM;
  }
  return HOM_OK;
}

int check_last() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    last_cuda_error() = e;
    return HOM_ERR_CUDA;
  }
  return HOM_OK;
}

// ---- autotuned launch plans, per (precision, grid, support) in this process ----
namespace {
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::map<TuneKey, PlanChoice>& tune_table() {
  static std::map<TuneKey, PlanChoice> t;
  return t;
}
std::mutex& tune_mu() {
  static std::mutex m;
  return m;
}
TuneKey tune_key(int pb, int d, const int* M, const int* N, int nc) {
  return TuneKey(pb, d, M[0], d > 1 ? M[1] : 1, d > 2 ? M[2] : 1, N[0], d > 1 ? N[1] : 1,
                 d > 2 ? N[2] : 1, nc > 0 ? nc : d);
}
}  // namespace

PlanChoice plan_choice(int pb, int d, const int* M, const int* N, int nc) {
  std::lock_guard<std::mutex> lk(tune_mu());
  auto it = tune_table().find(tune_key(pb, d, M, N, nc));
  if (it != tune_table().end()) return it->second;
  // defaults: two CTAs per SM in every pass; FP64 values take twice the registers
  return PlanChoice{pb == 8 ? 15 : 27, 110 * 1024, kThreads, true};
}

// Half spectrum on the grid M of the Fourier coefficients of a voxel-wise constant scalar
// coefficient a on the grid N (value a[k] on the cell of side 1/N centred at x = k/N): the cell
// integral of exp(-2 pi i n.x) (eq. (FT_def)) gives A^(n) = prod_a sinc(pi n_a / N_a)
// (F_N a)(n mod N), F_N the DFT of eq. (DFT) with its 1/|N|. F_N a comes from the library's
// forward transform on N; n mod N above the stored half of the last axis is read through
// Hermitian symmetry. Layout of `half`: M-grid lines (axes 0 .. d-2, row-major) x (M_last+1)/2.
int voxel_coefficients(hom_problem* P, const std::vector<double>& a,
                       std::vector<cpx<double>>& half) {
  const int d = P->d;
  const int* N = P->N;
  const int* M = P->M;
  long long nN = 1;
  for (int ax = 0; ax < d; ++ax) nN *= N[ax];
  const int nhN = (N[d - 1] + 1) / 2, mh = (M[d - 1] + 1) / 2;
  const long long nlN = nN / N[d - 1];
  Engine<double> eN;
  const PlanChoice pc = plan_choice(8, d, N, N);
  int st = eN.init(d, N, N, pc.budget, pc.rmax, pc.threads, pc.two_line);
  double* a_dev = nullptr;
  cpx<double>* s_dev = nullptr;
  if (st == HOM_OK) st = alloc((void**)&a_dev, sizeof(double) * nN);
  if (st == HOM_OK) st = alloc((void**)&s_dev, sizeof(cpx<double>) * nlN * nhN);
  std::vector<cpx<double>> sN((size_t)nlN * nhN);
  if (st == HOM_OK) {
    cudaMemcpy(a_dev, a.data(), sizeof(double) * nN, cudaMemcpyHostToDevice);
    eN.forward(a_dev, s_dev, 1, P->stream);
    if (cudaStreamSynchronize(P->stream) != cudaSuccess || check_last() != HOM_OK) st = HOM_ERR_CUDA;
    else cudaMemcpy(sN.data(), s_dev, sizeof(cpx<double>) * sN.size(), cudaMemcpyDeviceToHost);
  }
  if (a_dev) cudaFree(a_dev);
  if (s_dev) cudaFree(s_dev);
  eN.release();
  if (st != HOM_OK) return st;
  const double inv = 1.0 / (double)nN;
  const double pi = 3.14159265358979323846;
  // per-axis factors of the M-grid storage positions: n mod N and sinc(pi n / N)
  std::vector<int> pos[3];
  std::vector<double> sinc[3];
  for (int ax = 0; ax < d; ++ax) {
    pos[ax].resize(M[ax]);
    sinc[ax].resize(M[ax]);
    for (int j = 0; j < M[ax]; ++j) {
      const int n = j <= (M[ax] - 1) / 2 ? j : j - M[ax];
      pos[ax][j] = ((n % N[ax]) + N[ax]) % N[ax];
      const double t = pi * (double)n / (double)N[ax];
      sinc[ax][j] = n == 0 ? 1.0 : std::sin(t) / t;
    }
  }
  const long long nlM = (long long)half.size() / mh;
  for (long long l = 0; l < nlM; ++l) {
    // M-grid line l -> storage positions j_0 .. j_{d-2}
    int j[2] = {0, 0};
    if (d == 2) j[0] = (int)l;
    else { j[0] = (int)(l / M[1]); j[1] = (int)(l % M[1]); }
    double f = 1.0;
    for (int ax = 0; ax < d - 1; ++ax) f *= sinc[ax][j[ax]];
    for (int k = 0; k < mh; ++k) {
      const int ml = pos[d - 1][k];
      cpx<double> v;
      if (ml < nhN) {
        long long lN = d == 2 ? pos[0][j[0]] : (long long)pos[0][j[0]] * N[1] + pos[1][j[1]];
        v = sN[lN * nhN + ml];
      } else {  // X(m) = conj X(-m) for the real image
        const int q0 = (N[0] - pos[0][j[0]]) % N[0];
        long long lN = q0;
        if (d == 3) lN = (long long)q0 * N[1] + (N[1] - pos[1][j[1]]) % N[1];
        v = sN[lN * nhN + (N[d - 1] - ml)];
        v.y = -v.y;
      }
      const double c = f * sinc[d - 1][k] * inv;
      half[l * mh + k] = cpx<double>{v.x * c, v.y * c};
    }
  }
  return HOM_OK;
}

}  // namespace detail
}  // namespace hom

using namespace hom::detail;

namespace {
// Device address of a host pointer into page-locked memory (its mapping in the unified address
// space), or null for memory the device cannot address (pageable, or not host memory).
const void* mapped_host(const void* h) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) return at.devicePointer;
  return nullptr;
}

// Per-device set-up of the kernels: the register-DFT constants live in __constant__ memory and
// the shared-memory limits are function attributes, both state of the device that was current
// when they were set. Done once per device, with that device current.
constexpr int kMaxDevices = 64;
std::once_flag g_const_once[kMaxDevices];
cudaError_t g_const_err[kMaxDevices] = {};

cudaError_t device_setup() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::call_once(g_const_once[dev], [dev] {
    cudaError_t r = Ops<double>::upload_constants();
    if (r == cudaSuccess) r = Ops<float>::upload_constants();
    if (r == cudaSuccess) r = Ops<double>::prepare(3);
    if (r == cudaSuccess) r = Ops<float>::prepare(3);
    g_const_err[dev] = r;
  });
  return g_const_err[dev];
}
}  // namespace


extern "C" {

const char* hom_strerror(int s) {
  switch (s) {
    case HOM_OK: return "ok";
    case HOM_ERR_INVALID: return "invalid argument";
    case HOM_ERR_OOM: return "device out of memory";
    case HOM_ERR_UNSUPPORTED: return "unsupported combination";
    case HOM_ERR_NOT_CONVERGED: return "iteration limit reached before convergence";
    case HOM_ERR_CUDA: {
      static char buf[256];
      std::snprintf(buf, sizeof buf, "CUDA error: %s", cudaGetErrorString(last_cuda_error()));
      return buf;
    }
    case HOM_ERR_TIMEOUT: return "device wait timed out";
    case HOM_ERR_SCRATCH: return "problem too large for the static scratch of hom_apply_static";
    default: return "unknown status";
  }
}

long long hom_kernel_launches(void) { return launch_counter(); }

int hom_debug_fail_alloc(int n) {
  fail_countdown().store(n >= 0 ? (long long)n : -1LL);
  return HOM_OK;
}

int hom_debug_tma_stall(int on) {
  tma_debug_stall(on != 0);
  return HOM_OK;
}

int hom_profile_enable(int on) {
  ProfState& ps = prof_state();
  if (on) {
    ps.marks.clear();
    ps.used = 0;
  }
  ps.on = on != 0;
  return HOM_OK;
}

int hom_profile_read(double* ms, long long* launches, int nkinds) {
  if (!ms || !launches || nkinds < 1) return HOM_ERR_INVALID;
  ProfState& ps = prof_state();
  for (int k = 0; k < nkinds; ++k) {
    ms[k] = 0;
    launches[k] = 0;
  }
  for (auto& m : ps.marks) {
    if (m.first >= nkinds) continue;
    if (cudaEventSynchronize(m.second.second) != cudaSuccess) return HOM_ERR_CUDA;
    float t = 0;
    cudaEventElapsedTime(&t, m.second.first, m.second.second);
    ms[m.first] += t;
    launches[m.first] += 1;
  }
  return HOM_OK;
}

void hom_destroy(hom_problem* P) {
  if (!P) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  P->e64.release();
  P->e32.release();
  P->eN.release();
  if (P->SN) cudaFree(P->SN);
  if (P->yN) cudaFree(P->yN);
  if (P->d_phase) cudaFree(P->d_phase);
  if (P->d_table) cudaFree(P->d_table);
  if (P->d_inv) cudaFree(P->d_inv);
  if (P->S) cudaFree(P->S);
  if (P->vbase) cudaFree(P->vbase);
  for (auto& v : P->fvec)
    if (v) cudaFree(v);
  if (P->partials) cudaFree(P->partials);
  if (P->d_hist) cudaFree(P->d_hist);
  if (P->counter) cudaFree(P->counter);
  if (P->d_sc) cudaFree(P->d_sc);
  if (P->d_aux) cudaFree(P->d_aux);
  if (P->d_sc2) cudaFree(P->d_sc2);
  if (P->h_sc) cudaFreeHost(P->h_sc);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  delete P;
  cudaSetDevice(cur);
}

int hom_grid(const hom_problem* P, int* M_out, long long* nodes) {
  if (!P) return HOM_ERR_INVALID;
  if (M_out)
    for (int a = 0; a < P->d; ++a) M_out[a] = P->M[a];
  if (nodes) *nodes = P->nodes;
  return HOM_OK;
}

int hom_bounds(const hom_problem* P, double* cA, double* CA) {
  if (!P) return HOM_ERR_INVALID;
  if (cA) *cA = P->cA;
  if (CA) *CA = P->CA;
  return HOM_OK;
}

int hom_create(int d, const int* N, const hom_material* A, int integration, int precision,
               void* stream, hom_problem** out) {
  if (!out || !N || !A) return HOM_ERR_INVALID;
  *out = nullptr;
  if (d != 2 && d != 3) return HOM_ERR_INVALID;
  if (integration != HOM_APPROX && integration != HOM_EXACT) return HOM_ERR_INVALID;
  if (precision != HOM_FP64 && precision != HOM_FP32_REFINED) return HOM_ERR_INVALID;
  for (int a = 0; a < d; ++a)
    if (N[a] < 3 || N[a] % 2 == 0 || N[a] > kMaxAxis) return HOM_ERR_INVALID;
  if (integration == HOM_APPROX && A->kind == HOM_A_FOURIER) return HOM_ERR_INVALID;
  // linear elasticity: symmetric strain fields of nc = d (d + 1) / 2 components (Mandel),
  // sampled stiffness (GaNi), FP64 or FP32 inner solves with FP64 refinement
  const bool elastic = A->kind == HOM_A_STIFFNESS;
  const int nc = elastic ? d * (d + 1) / 2 : d;
  if (elastic && integration != HOM_APPROX) return HOM_ERR_UNSUPPORTED;
  // exact integration of an image (voxel-wise constant coefficients): scalar coefficients only
  const bool voxel_ga = integration == HOM_EXACT && A->kind != HOM_A_FOURIER;
  if (voxel_ga) {
    if (A->kind != HOM_A_PHASE && A->kind != HOM_A_SCALAR) return HOM_ERR_INVALID;
    if (A->kind == HOM_A_PHASE) {
      if (!A->table || A->nphase < 1) return HOM_ERR_INVALID;
      for (int p = 0; p < A->nphase; ++p) {
        const double* t = A->table + (size_t)p * d * d;
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j)
            if ((i != j && t[i * d + j] != 0.0) || (i == j && t[i * d + j] != t[0]))
              return HOM_ERR_UNSUPPORTED;
      }
    }
  }

  {
    const cudaError_t ce = device_setup();
    if (ce != cudaSuccess) {
      last_cuda_error() = ce;
      return HOM_ERR_CUDA;
    }
  }

  hom_problem* P = new hom_problem();
  P->d = d;
  P->nc = nc;
  P->integration = integration;
  P->precision = precision;
  P->stream = (cudaStream_t)stream;
  cudaGetDevice(&P->device);
  for (int a = 0; a < d; ++a) {
    P->N[a] = N[a];
    P->M[a] = N[a];
  }
  if (integration == HOM_EXACT) {
    for (int a = 0; a < d; ++a) {
      const int m = A->M[a] > 0 ? A->M[a] : 2 * N[a] - 1;
      if (m < 2 * N[a] - 1 || m % 2 == 0 || m > kMaxAxis) {
        delete P;
        return HOM_ERR_INVALID;
      }
      P->M[a] = m;
    }
  }
  P->nodes = 1;
  for (int a = 0; a < d; ++a) P->nodes *= P->M[a];
  if (P->nodes > kMaxNodes) {
    delete P;
    return HOM_ERR_INVALID;
  }
  const long long nodes = P->nodes;
  int st;
  long long nN = 1;  // nodes of the image grid N
  for (int a = 0; a < d; ++a) nN *= P->N[a];
  std::vector<double> voxel;  // voxel_ga: the image's scalar coefficient on the N grid

  // ---- coefficients ----
  if (voxel_ga) {
    if (!A->data || (A->kind == HOM_A_PHASE && A->index_bytes != 1 && A->index_bytes != 2)) {
      delete P;
      return HOM_ERR_INVALID;
    }
    voxel.resize(nN);
    if (A->kind == HOM_A_SCALAR) {
      if (A->data_on_device)
        cudaMemcpy(voxel.data(), A->data, sizeof(double) * nN, cudaMemcpyDeviceToHost);
      else
        std::memcpy(voxel.data(), A->data, sizeof(double) * nN);
    } else {
      std::vector<unsigned char> ph((size_t)nN * A->index_bytes);
      if (A->data_on_device)
        cudaMemcpy(ph.data(), A->data, ph.size(), cudaMemcpyDeviceToHost);
      else
        std::memcpy(ph.data(), A->data, ph.size());
      for (long long g = 0; g < nN; ++g) {
        const int i = A->index_bytes == 1 ? ph[g] : ((const uint16_t*)ph.data())[g];
        if (i >= A->nphase) { delete P; return HOM_ERR_INVALID; }
        voxel[g] = A->table[(size_t)i * d * d];
      }
    }
    double lo = 1e300, hi = -1e300;
    for (double v : voxel) {
      lo = std::min(lo, v);
      hi = std::max(hi, v);
    }
    if (!(lo > 0)) { delete P; return HOM_ERR_INVALID; }
    P->cA = lo;
    P->CA = hi;
    P->mat_kind = MAT_FIELD;
  } else if (A->kind == HOM_A_PHASE || elastic) {
    if (!A->data || !A->table || A->nphase < 1 || (A->index_bytes != 1 && A->index_bytes != 2) ||
        (A->index_bytes == 1 && A->nphase > 256)) {
      delete P;
      return HOM_ERR_INVALID;
    }
    // tables of d x d conductivities or nc x nc Mandel stiffnesses (never taken as isotropic)
    bool iso = !elastic;
    double lo = 1e300, hi = -1e300;
    for (int p = 0; p < A->nphase; ++p) {
      const double* t = A->table + (size_t)p * nc * nc;
      double l, h;
      if (!spd_eigs(t, nc, &l, &h)) {
        delete P;
        return HOM_ERR_INVALID;
      }
      lo = std::min(lo, l);
      hi = std::max(hi, h);
      for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j)
          if ((i != j && t[i * nc + j] != 0.0) || (i == j && t[i * nc + j] != t[0])) iso = false;
    }
    P->cA = lo;
    P->CA = hi;
    P->mat_kind = iso ? MAT_PHASE_ISO : MAT_PHASE_TENSOR;
    P->index_bytes = A->index_bytes;
    P->nphase = A->nphase;
    std::vector<double> tab;
    if (iso) {
      for (int p = 0; p < A->nphase; ++p) tab.push_back(A->table[(size_t)p * d * d]);
    } else {
      tab.assign(A->table, A->table + (size_t)A->nphase * nc * nc);
    }
    if ((st = alloc((void**)&P->d_table, sizeof(double) * tab.size())) != HOM_OK) { hom_destroy(P); return st; }
    // 16 zero bytes past the end: kernels may read the phase indices in aligned words
    if ((st = alloc(&P->d_phase, (size_t)nodes * A->index_bytes + 16)) != HOM_OK) { hom_destroy(P); return st; }
    cudaMemset((char*)P->d_phase + (size_t)nodes * A->index_bytes, 0, 16);
    cudaMemcpy(P->d_table, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(P->d_phase, A->data, (size_t)nodes * A->index_bytes,
               A->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    // phase indices must address the table
    if (!A->data_on_device) {
      for (long long g = 0; g < nodes; ++g) {
        const int ph = A->index_bytes == 1 ? ((const uint8_t*)A->data)[g] : ((const uint16_t*)A->data)[g];
        if (ph >= A->nphase) { hom_destroy(P); return HOM_ERR_INVALID; }
      }
    }
  } else if (A->kind == HOM_A_SCALAR) {
    if (!A->data) { delete P; return HOM_ERR_INVALID; }
    P->mat_kind = MAT_FIELD;
    if ((st = alloc((void**)&P->e64.field, sizeof(double) * nodes)) != HOM_OK) { hom_destroy(P); return st; }
    cudaMemcpy(P->e64.field, A->data, sizeof(double) * nodes,
               A->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    {
      std::vector<double> hcopy;
      const double* a = (const double*)A->data;
      if (A->data_on_device) {
        hcopy.resize(nodes);
        cudaMemcpy(hcopy.data(), A->data, sizeof(double) * nodes, cudaMemcpyDeviceToHost);
        a = hcopy.data();
      }
      double lo = 1e300, hi = -1e300;
      for (long long g = 0; g < nodes; ++g) {
        lo = std::min(lo, a[g]);
        hi = std::max(hi, a[g]);
      }
      if (!(lo > 0)) { hom_destroy(P); return HOM_ERR_INVALID; }
      P->cA = lo;
      P->CA = hi;
    }
  } else if (A->kind == HOM_A_FOURIER) {
    if (!A->data) { delete P; return HOM_ERR_INVALID; }
    P->mat_kind = MAT_FIELD;
  } else {
    delete P;
    return HOM_ERR_INVALID;
  }
  if (A->cA > 0) P->cA = A->cA;
  if (A->CA > 0) P->CA = A->CA;
  if (!(P->cA > 0 && P->CA >= P->cA)) { hom_destroy(P); return HOM_ERR_INVALID; }

  // ---- plans ----
  {
    const PlanChoice pc = plan_choice(8, d, P->M, P->N, nc);
    if ((st = P->e64.init(d, P->M, P->N, pc.budget, pc.rmax, pc.threads, pc.two_line, nc)) != HOM_OK) { hom_destroy(P); return st; }
  }
  if (precision == HOM_FP32_REFINED) {
    const PlanChoice pc = plan_choice(4, d, P->M, P->N, nc);
    if ((st = P->e32.init(d, P->M, P->N, pc.budget, pc.rmax, pc.threads, pc.two_line, nc)) != HOM_OK) { hom_destroy(P); return st; }
  }

  // ---- buffers ----
  P->S_bytes = sizeof(cpx<double>) * (size_t)P->nc * P->e64.g.scs;
  if ((st = alloc(&P->S, P->S_bytes)) != HOM_OK) { hom_destroy(P); return st; }
  if ((st = alloc((void**)&P->vbase, sizeof(double) * 5 * P->nc * nodes)) != HOM_OK) { hom_destroy(P); return st; }
  for (int i = 0; i < 5; ++i) P->vec[i] = P->vbase + (size_t)i * P->nc * nodes;
  if (precision == HOM_FP32_REFINED)
    for (int i = 0; i < 4; ++i)
      if ((st = alloc((void**)&P->fvec[i], sizeof(float) * P->nc * nodes)) != HOM_OK) { hom_destroy(P); return st; }
  P->red_grid = (int)std::min<long long>((nodes * P->nc + kThreads - 1) / kThreads, 152 * 8);
  long long maxblocks = std::max<long long>(P->red_grid, (P->e64.g.nlines + 1) / 2 + 1);
  // k_energy reduces nc + 1 values per CTA (energy and the nc flux components)
  P->npartials = (size_t)maxblocks * (size_t)std::max(4, P->nc + 1);
  if ((st = alloc((void**)&P->partials, sizeof(double) * P->npartials)) != HOM_OK) { hom_destroy(P); return st; }
  if ((st = alloc((void**)&P->counter, sizeof(unsigned) * 4)) != HOM_OK) { hom_destroy(P); return st; }
  cudaMemset(P->counter, 0, sizeof(unsigned) * 4);
  if ((st = alloc((void**)&P->d_sc, sizeof(Scalars))) != HOM_OK) { hom_destroy(P); return st; }
  if ((st = alloc((void**)&P->d_aux, sizeof(Scalars))) != HOM_OK) { hom_destroy(P); return st; }
  if ((st = alloc((void**)&P->d_sc2, sizeof(Scalars))) != HOM_OK) { hom_destroy(P); return st; }
  if (cudaMallocHost((void**)&P->h_sc, sizeof(Scalars)) != cudaSuccess) { hom_destroy(P); return HOM_ERR_OOM; }
  cudaEventCreate(&P->ev0);
  cudaEventCreate(&P->ev1);

  P->e64.mat = make_view<double>(P, P->e64.field, P->d_table);

  // ---- Ga: A_M^k = sum_n omega_M^{kn} A^(n) (eq. (Ga_exact_integration)) ----
  if (A->kind == HOM_A_FOURIER || voxel_ga) {
    if ((st = alloc((void**)&P->e64.field, sizeof(double) * nodes)) != HOM_OK) { hom_destroy(P); return st; }
    const int D = d;
    const long long mh = P->e64.g.nh;
    const long long nl = P->e64.g.nlines;
    std::vector<cpx<double>> half((size_t)nl * mh);
    const int mlast = P->M[D - 1];
    if (voxel_ga) {
      if ((st = voxel_coefficients(P, voxel, half)) != HOM_OK) { hom_destroy(P); return st; }
    } else {
      std::vector<double> full((size_t)nodes * 2);
      if (A->data_on_device)
        cudaMemcpy(full.data(), A->data, sizeof(double) * 2 * nodes, cudaMemcpyDeviceToHost);
      else
        std::memcpy(full.data(), A->data, sizeof(double) * 2 * nodes);
      for (long long l = 0; l < nl; ++l)
        for (long long k = 0; k < mh; ++k) {
          half[l * mh + k].x = full[2 * (l * mlast + k)];
          half[l * mh + k].y = full[2 * (l * mlast + k) + 1];
        }
    }
    cudaMemcpy(P->S, half.data(), sizeof(cpx<double>) * half.size(), cudaMemcpyHostToDevice);
    P->e64.inverse((cpx<double>*)P->S, P->e64.field, 1, P->stream);
    if (cudaStreamSynchronize(P->stream) != cudaSuccess || check_last() != HOM_OK) {
      hom_destroy(P);
      return HOM_ERR_CUDA;
    }
    P->e64.mat = make_view<double>(P, P->e64.field, P->d_table);
  }
  if (precision == HOM_FP32_REFINED) {
    if (P->d_table) {
      const size_t ntab = (P->mat_kind == MAT_PHASE_ISO) ? (size_t)P->nphase : (size_t)P->nphase * nc * nc;
      std::vector<double> h(ntab);
      std::vector<float> hf(ntab);
      cudaMemcpy(h.data(), P->d_table, sizeof(double) * ntab, cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < ntab; ++i) hf[i] = (float)h[i];
      if ((st = alloc((void**)&P->e32.table, sizeof(float) * ntab)) != HOM_OK) { hom_destroy(P); return st; }
      cudaMemcpy(P->e32.table, hf.data(), sizeof(float) * ntab, cudaMemcpyHostToDevice);
    }
    if (P->mat_kind == MAT_FIELD) {
      if ((st = alloc((void**)&P->e32.field, sizeof(float) * nodes)) != HOM_OK) { hom_destroy(P); return st; }
      std::vector<double> h(nodes);
      std::vector<float> hf(nodes);
      cudaMemcpy(h.data(), P->e64.field, sizeof(double) * nodes, cudaMemcpyDeviceToHost);
      for (long long g = 0; g < nodes; ++g) hf[g] = (float)h[g];
      cudaMemcpy(P->e32.field, hf.data(), sizeof(float) * nodes, cudaMemcpyHostToDevice);
    }
    P->e32.mat = make_view<float>(P, P->e32.field, P->e32.table);
  }
  if (check_last() != HOM_OK) { hom_destroy(P); return HOM_ERR_CUDA; }
  *out = P;
  return HOM_OK;
}

int hom_apply(hom_problem* P, int op, const double* E, const double* x_dev, double* y_dev) {
  if (!P || !x_dev || !y_dev) return HOM_ERR_INVALID;
  const bool fp32 = (op & HOM_OP_FP32) != 0;
  const bool x_host = (op & HOM_OP_X_HOST) != 0, y_host = (op & HOM_OP_Y_HOST) != 0;
  op &= ~(HOM_OP_FP32 | HOM_OP_X_HOST | HOM_OP_Y_HOST);
  if (x_host || y_host) {
    if (op < HOM_OP_AFFINE || op > HOM_OP_EM) return HOM_ERR_INVALID;
    // page-locked host memory through its device mapping; anything else staged through the
    // free solver vector vec[4] (the operator may run in place)
    const size_t bytes = sizeof(double) * (size_t)P->nc * (size_t)P->nodes;
    double* stage = P->vec[4];
    const double* xd = x_dev;
    double* yd = y_dev;
    if (x_host) {
      xd = static_cast<const double*>(mapped_host(x_dev));
      if (!xd) {
        HOM_CUDA(cudaMemcpyAsync(stage, x_dev, bytes, cudaMemcpyHostToDevice, P->stream));
        xd = stage;
      }
    }
    bool y_staged = false;
    if (y_host) {
      yd = static_cast<double*>(const_cast<void*>(mapped_host(y_dev)));
      if (!yd) {
        yd = stage;
        y_staged = true;
      }
    }
    int rc = hom_apply(P, op | (fp32 ? HOM_OP_FP32 : 0), E, xd, yd);
    if (rc) return rc;
    if (y_staged) HOM_CUDA(cudaMemcpyAsync(y_dev, stage, bytes, cudaMemcpyDeviceToHost, P->stream));
    if (y_host) HOM_CUDA(cudaStreamSynchronize(P->stream));
    return check_last();
  }
  if (op < HOM_OP_AFFINE || op > HOM_OP_EM) return HOM_ERR_INVALID;
  if (op == HOM_OP_AFFINE && !E) return HOM_ERR_INVALID;
  if (op == HOM_OP_EM && P->integration == HOM_EXACT) return HOM_ERR_UNSUPPORTED;
  if (fp32 && P->precision != HOM_FP32_REFINED) return HOM_ERR_UNSUPPORTED;
  OpArgs args{};
  for (int a = 0; a < P->nc; ++a) args.E[a] = E ? E[a] : 0.0;
  args.omega = std::sqrt(P->cA * P->CA);
  const int pre = op == HOM_OP_AFFINE ? PRE_AFFINE : op == HOM_OP_LINEAR ? PRE_LINEAR
                : op == HOM_OP_PROJECT ? PRE_IDENT : PRE_EM;
  const int mode = op == HOM_OP_EM ? PROJ_EM : PROJ_GAMMA;
  if (fp32) {
    const long long len = (long long)P->nc * P->nodes;
    Ops<float>::convert_in(x_dev, P->fvec[0], len, P->stream);
    Fields<float> f{};
    f.xin = P->fvec[0];
    f.out = P->fvec[1];
    f.cs = P->nodes;
    P->e32.apply(pre, mode, POST_STORE, f, (cpx<float>*)P->S, nullptr, args, nullptr, nullptr, 0,
                 P->stream);
    Ops<float>::convert_out(P->fvec[1], y_dev, len, P->stream);
    return check_last();
  }
  Fields<double> f{};
  f.xin = x_dev;
  f.out = y_dev;
  f.cs = P->nodes;
  P->e64.apply(pre, mode, POST_STORE, f, (cpx<double>*)P->S, nullptr, args, nullptr, nullptr, 0,
               P->stream);
  return check_last();
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// solver drivers
// ---------------------------------------------------------------------------------------
namespace hom {
namespace detail {

int poll(hom_problem* P, Scalars* dst) {
  HOM_CUDA(cudaMemcpyAsync(P->h_sc, dst, sizeof(Scalars), cudaMemcpyDeviceToHost, P->stream));
  HOM_CUDA(cudaStreamSynchronize(P->stream));
  return HOM_OK;
}

int upload_scalars(hom_problem* P, Scalars* dst, const Scalars& s) {
  *P->h_sc = s;
  HOM_CUDA(cudaMemcpyAsync(dst, P->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, P->stream));
  HOM_CUDA(cudaStreamSynchronize(P->stream));
  return HOM_OK;
}

// (A(E + x), E + x) and <A(E + x)> into P->d_aux
int energy_eval(hom_problem* P, const double* E, const double* x, double* en, double* flux) {
  Scalars s{};
  for (int a = 0; a < P->nc; ++a) s.E[a] = E[a];
  int st = upload_scalars(P, P->d_aux, s);
  if (st) return st;
  Ops<double>::energy(P->nc, x, P->nodes, P->e64.mat, P->d_aux, P->partials, P->counter,
                      P->red_grid, P->stream);
  if ((st = check_last())) return st;
  if ((st = poll(P, P->d_aux))) return st;
  if (en) *en = P->h_sc->energy;
  if (flux)
    for (int a = 0; a < P->nc; ++a) flux[a] = P->h_sc->flux[a];
  return HOM_OK;
}

// ||G A (E + x)|| (the residual b - C x up to sign) into P->d_aux; y is scratch
double true_residual(hom_problem* P, const double* E, const double* x, double* y) {
  Scalars s{};
  for (int a = 0; a < P->nc; ++a) s.E[a] = E[a];
  if (upload_scalars(P, P->d_aux, s)) return -1;
  Fields<double> f{};
  f.xin = x;
  f.out = y;
  f.cs = P->nodes;
  OpArgs args{};
  P->e64.apply(PRE_AFFINE, PROJ_GAMMA, POST_STORE, f, (cpx<double>*)P->S, P->d_aux, args,
               P->partials, P->counter, 0, P->stream);
  if (poll(P, P->d_aux)) return -1;
  return P->h_sc->nb;
}

// the N-grid engine, spectrum and field of an exact-integration problem (first use)
int ensure_ngrid(hom_problem* P) {
  if (P->eN.ready && P->SN && P->yN) return HOM_OK;
  const PlanChoice pc = plan_choice(8, P->d, P->N, P->N);
  int st = HOM_OK;
  if (!P->eN.ready) {
    st = P->eN.init(P->d, P->N, P->N, pc.budget, pc.rmax, pc.threads, pc.two_line);
    if (st != HOM_OK) {
      P->eN.release();
      P->eN.ready = false;
      return st;
    }
  }
  long long nN = 1;
  for (int a = 0; a < P->d; ++a) nN *= P->N[a];
  if (!P->SN && (st = alloc(&P->SN, sizeof(cpx<double>) * (size_t)P->d * P->eN.g.scs)) != HOM_OK)
    return st;
  if (!P->yN && (st = alloc((void**)&P->yN, sizeof(double) * (size_t)P->d * nN)) != HOM_OK)
    return st;
  return HOM_OK;
}

// y (N grid) = samples of the trigonometric polynomial of order N with values x on the solve
// grid M: F_M (unscaled), the coefficients of Z_N times 1/|M|, F_N^{-1} (eq. (DFT))
int restrict_field(hom_problem* P, const double* x, double* y) {
  const int d = P->d;
  cudaStream_t st = P->stream;
  if (P->integration != HOM_EXACT) {
    if (x != y)
      HOM_CUDA(cudaMemcpyAsync(y, x, sizeof(double) * P->nc * P->nodes, cudaMemcpyDeviceToDevice, st));
    return check_last();
  }
  int rc = ensure_ngrid(P);
  if (rc) return rc;
  P->e64.forward(x, (cpx<double>*)P->S, d, st);
  const PassGeom& gm = P->e64.g;
  const PassGeom& gn = P->eN.g;
  const int n1 = d == 3 ? gn.n[1] : 1, m1 = d == 3 ? gm.n[1] : 1;
  Ops<double>::crop_spectrum((const cpx<double>*)P->S, (cpx<double>*)P->SN, d, gn.n[0], n1, gn.nh,
                             gm.n[0], m1, gm.nh, 1.0 / (double)gm.nodes, gn.scs, gm.scs, st);
  P->eN.inverse((cpx<double>*)P->SN, y, d, st);
  return check_last();
}

// The corrector output of a session from the device field src on the solve grid: on the
// device or the host (HOM_OUT_HOST), on the solve grid or as N-grid samples (HOM_OUT_NGRID,
// exact integration). Synchronises the stream.
int write_corrector(hom_problem* P, const double* src, double* out) {
  const int f = P->sv.out_flags;
  const bool ngrid = (f & HOM_OUT_NGRID) && P->integration == HOM_EXACT;
  const bool host = (f & HOM_OUT_HOST) != 0;
  long long n = P->nodes;
  if (ngrid) {
    n = 1;
    for (int a = 0; a < P->d; ++a) n *= P->N[a];
  }
  const size_t bytes = sizeof(double) * (size_t)P->nc * (size_t)n;
  const double* res = src;
  if (ngrid) {
    int rc = ensure_ngrid(P);
    if (rc) return rc;
    double* dst = host ? P->yN : out;
    if ((rc = restrict_field(P, src, dst))) return rc;
    res = dst;
  }
  if (host)
    HOM_CUDA(cudaMemcpyAsync(out, res, bytes, cudaMemcpyDeviceToHost, P->stream));
  else if (res != out)
    HOM_CUDA(cudaMemcpyAsync(out, res, bytes, cudaMemcpyDeviceToDevice, P->stream));
  HOM_CUDA(cudaStreamSynchronize(P->stream));
  return check_last();
}

}  // namespace detail
}  // namespace hom

// ---------------------------------------------------------------------------------------
// solve sessions: begin (validation, x_0, r_0 = b), iterate (enqueue steps), end (outputs)
// ---------------------------------------------------------------------------------------
namespace hom {
namespace detail {

int solve_stop_mode(int solver, int stop) {
  if (stop == HOM_STOP_DEFAULT) return solver == HOM_EYRE_MILTON ? HOM_STOP_INCREMENT : HOM_STOP_RESIDUAL;
  return stop;
}

// enqueue one iteration of the active solver (Algorithms 1-4); kernels exit early once the
// device stopping flag is set
void enqueue_step(hom_problem* P) {
  SolveState& S_ = P->sv;
  const long long nodes = P->nodes;
  cpx<double>* S = (cpx<double>*)P->S;
  cudaStream_t st = P->stream;
  OpArgs args{};
  double* x = P->vec[0];
  double* r = P->vec[2];
  double* p = P->vec[3];
  Fields<double> f{};
  f.cs = nodes;
  switch (S_.solver) {
    case HOM_RICHARDSON:
      f.x = P->vec[0];  // x_m / x_{m-1} alternate between vec[0] and vec[1]
      P->e64.apply(PRE_AFFINE, PROJ_GAMMA, POST_RICH, f, S, P->d_sc, args, P->partials,
                   P->counter, 0, st);
      break;
    case HOM_CG: {
      // Algorithm 2 with the vector update fused into the operator passes (as the FP32 inner
      // solves do): the pre-operator pass forms p = r + beta p, A p and (p, A p) = (p, C p) (p
      // lies in the range of G), then alpha; the inverse pass updates x and r and forms (r, r)
      f.xin = r;
      f.p = p;
      Fields<double> fi = f;
      fi.x = x;
      fi.r = r;
      P->e64.apply2(PRE_CG_DOT, PROJ_GAMMA, POST_CG_FUSED, f, fi, S, P->d_sc, args, P->partials,
                    P->counter, 0, st);
      break;
    }
    case HOM_CHEBYSHEV: {
      f.xin = p;
      Fields<double> fi = f;
      fi.p = p;
      fi.r = r;
      fi.x = x;
      P->e64.apply2(PRE_LINEAR, PROJ_GAMMA, POST_CHEB, f, fi, S, P->d_sc, args, P->partials,
                    P->counter, 0, st);
      break;
    }
    default: {  // Eyre-Milton
      f.xin = x;
      Fields<double> fi = f;
      fi.x = x;
      P->e64.apply2(PRE_EM, PROJ_EM, POST_EM, f, fi, S, P->d_sc, args, P->partials, P->counter,
                    0, st);
      break;
    }
  }
  S_.issued += 1;
}

}  // namespace detail
}  // namespace hom

namespace hom {
namespace detail {

// the vectors of the FP32 inner CG in potential coordinates: u, r, p in fvec[0..2] (each
// holds the one-component half spectrum, at most half of its d |N| floats)
PotVecs<float> pot_vecs(hom_problem* P) {
  return PotVecs<float>{(cpx<float>*)P->fvec[0], (cpx<float>*)P->fvec[1],
                        (cpx<float>*)P->fvec[2]};
}

// r = b - C x = -G A (E + x) in FP64 into vec[2]; returns ||r|| (host synchronises)
int refine_residual(hom_problem* P, double* res) {
  SolveState& S_ = P->sv;
  Scalars s{};
  for (int a = 0; a < P->nc; ++a) s.E[a] = S_.E[a];
  int rc = upload_scalars(P, P->d_aux, s);
  if (rc) return rc;
  Fields<double> f{};
  f.xin = P->vec[0];
  f.out = P->vec[2];
  f.cs = P->nodes;
  OpArgs args{};
  P->e64.apply(PRE_AFFINE, PROJ_GAMMA, POST_STORE, f, (cpx<double>*)P->S, P->d_aux, args,
               P->partials, P->counter, 1, P->stream);
  if ((rc = check_last()) || (rc = poll(P, P->d_aux))) return rc;
  *res = P->h_sc->nb;
  return HOM_OK;
}

// start an FP32 inner solve of C d = r (Algorithm 2 or 3 on the FP32 operator)
int refine_start_inner(hom_problem* P) {
  SolveState& S_ = P->sv;
  Scalars s{};
  s.tol = S_.inner_tol;
  s.maxit = S_.inner_maxit;
  s.stop = HOM_STOP_RESIDUAL;
  if (S_.solver == HOM_CHEBYSHEV) {
    s.cheb_c = 0.5 * (P->CA - P->cA);
    s.cheb_d = 0.5 * (P->cA + P->CA);
    s.alpha = 1.0 / s.cheb_d;
    s.beta = -0.5 * (s.cheb_c / s.cheb_d) * (s.cheb_c / s.cheb_d);
  }
  s.pot_cheb = S_.pot && S_.solver == HOM_CHEBYSHEV;
  int rc = upload_scalars(P, P->d_sc2, s);
  if (rc) return rc;
  if (S_.pot) {
    // r = D* r_field in potential coordinates (from the FP32 rounding of the FP64 residual)
    const long long n3 = (long long)P->nc * P->nodes;
    Ops<float>::convert_in(P->vec[2], P->fvec[3], n3, P->stream);
    P->e32.pot_init(P->fvec[3], pot_vecs(P), (cpx<float>*)P->S, P->d_sc2, P->partials,
                    P->counter, P->stream);
    return check_last();
  }
  const long long len = (long long)P->nc * P->nodes;
  Ops<float>::demote(P->vec[2], P->fvec[1], P->fvec[2], P->fvec[0], len, P->nodes, P->d_sc2,
                     P->partials, P->counter, P->red_grid, P->stream);
  if (S_.solver == HOM_CHEBYSHEV) {
    // demote zeroes beta; restore Algorithm 3's initial coefficients
    Scalars* h = P->h_sc;
    if ((rc = poll(P, P->d_sc2))) return rc;
    h->alpha = s.alpha;
    h->beta = s.beta;
    h->cheb_c = s.cheb_c;
    h->cheb_d = s.cheb_d;
    Scalars copy = *h;
    if ((rc = upload_scalars(P, P->d_sc2, copy))) return rc;
  }
  return check_last();
}

void refine_enqueue_inner(hom_problem* P) {
  if (P->sv.pot) {
    P->e32.pot_step(pot_vecs(P), (cpx<float>*)P->S, P->d_sc2, P->partials, P->counter,
                    P->stream, nullptr, 1, P->sv.solver == HOM_CHEBYSHEV);
    return;
  }
  const long long nodes = P->nodes;
  cpx<float>* S = (cpx<float>*)P->S;
  float* x = P->fvec[0];
  float* r = P->fvec[1];
  float* p = P->fvec[2];
  OpArgs args{};
  Fields<float> f{};
  f.cs = nodes;
  if (P->sv.solver == HOM_CG) {
    // the CG step with the vector update fused into the operator passes (PRE_CG_DOT computes
    // (p, A p) and alpha, POST_CG_FUSED updates x and r and forms (r, r) and beta)
    f.xin = r;
    f.p = p;
    Fields<float> fi = f;
    fi.x = x;
    fi.r = r;
    P->e32.apply2(PRE_CG_DOT, PROJ_GAMMA, POST_CG_FUSED, f, fi, S, P->d_sc2, args, P->partials,
                  P->counter, 0, P->stream);
  } else {
    f.xin = p;
    Fields<float> fi = f;
    fi.p = p;
    fi.r = r;
    fi.x = x;
    P->e32.apply2(PRE_LINEAR, PROJ_GAMMA, POST_CHEB, f, fi, S, P->d_sc2, args, P->partials,
                  P->counter, 0, P->stream);
  }
}

// after an inner solve stopped: x += d (FP64), new FP64 residual, stopping test
int refine_outer_update(hom_problem* P) {
  SolveState& S_ = P->sv;
  const long long len = (long long)P->nc * P->nodes;
  int rc = poll(P, P->d_sc2);
  if (rc) return rc;
  S_.inner_total += P->h_sc->it;
  // x += G d: the FP32 correction carries round-off outside the conforming space E (Section
  // 4.4); C does not see that part but the energy does, so it is projected out in FP64. In
  // potential coordinates d = D u is formed first (into fvec[3]).
  const float* dfield = P->fvec[0];
  if (S_.pot) {
    P->e32.pot_field(pot_vecs(P), (cpx<float>*)P->S, P->d_sc2, P->fvec[3], P->stream);
    dfield = P->fvec[3];
  }
  Ops<float>::convert_out(dfield, P->vec[4], len, P->stream);
  Fields<double> f{};
  f.xin = P->vec[4];
  f.x = P->vec[0];
  f.cs = P->nodes;
  Fields<double> ff = f;
  ff.x = nullptr;
  OpArgs args{};
  P->e64.apply2(PRE_IDENT, PROJ_GAMMA, POST_ADD, ff, f, (cpx<double>*)P->S, nullptr, args,
                nullptr, nullptr, 0, P->stream);
  S_.matvecs += 1;
  if ((rc = refine_residual(P, &S_.res))) return rc;
  S_.outer_hist.push_back(S_.res);
  S_.outer_it += 1;
  if (S_.res <= S_.tol * S_.nb) {
    S_.finished = true;
    S_.converged = true;
  } else if (S_.outer_it >= S_.maxit) {
    S_.finished = true;
  } else {
    rc = refine_start_inner(P);
  }
  return rc;
}

int refine_begin(hom_problem* P) {
  SolveState& S_ = P->sv;
  const long long len = (long long)P->nc * P->nodes;
  HOM_CUDA(cudaEventRecord(P->ev0, P->stream));
  HOM_CUDA(cudaMemsetAsync(P->vec[0], 0, sizeof(double) * len, P->stream));
  int rc = refine_residual(P, &S_.nb);
  if (rc) return rc;
  S_.res = S_.nb;
  S_.matvecs = 1;
  if (S_.nb == 0.0) {
    S_.finished = true;
    S_.converged = true;
    return HOM_OK;
  }
  return refine_start_inner(P);
}

}  // namespace detail
}  // namespace hom

static int solve_begin_impl(hom_problem* P, const double* E, int solver, double tol,
                            const hom_opts* opts) {
  if (solver < HOM_RICHARDSON || solver > HOM_EYRE_MILTON) return HOM_ERR_INVALID;
  hom_opts o{};
  if (opts) o = *opts;
  if (o.fixed_iters <= 0 && !(tol > 0)) return HOM_ERR_INVALID;
  if (solver == HOM_EYRE_MILTON && P->integration == HOM_EXACT) return HOM_ERR_UNSUPPORTED;
  const int stop = solve_stop_mode(solver, o.stop);
  if ((solver == HOM_CG || solver == HOM_CHEBYSHEV) && stop == HOM_STOP_INCREMENT) return HOM_ERR_UNSUPPORTED;
  if (solver == HOM_EYRE_MILTON && stop == HOM_STOP_RESIDUAL) return HOM_ERR_UNSUPPORTED;
  const int d = P->nc;  // components of the fields and of E
  const long long nodes = P->nodes;
  const long long len = (long long)d * nodes;
  const double cA = o.cA > 0 ? o.cA : P->cA;
  const double CA = o.CA > 0 ? o.CA : P->CA;
  SolveState& S_ = P->sv;
  S_ = SolveState{};
  S_.active = true;
  S_.solver = solver;
  S_.stop = stop;
  S_.fixed = o.fixed_iters > 0;
  S_.maxit = o.fixed_iters > 0 ? o.fixed_iters : (o.maxit > 0 ? o.maxit : 100000);
  S_.check = o.check_every > 0 ? o.check_every : 8;
  S_.out_flags = o.out_flags;
  for (int a = 0; a < d; ++a) S_.E[a] = E[a];
  double nE = 0;
  for (int a = 0; a < d; ++a) nE += E[a] * E[a];
  nE = std::sqrt(nE);
  S_.nE = nE;
  if (P->precision == HOM_FP32_REFINED) {
    if (solver != HOM_CG && solver != HOM_CHEBYSHEV) return HOM_ERR_UNSUPPORTED;
    S_.refined = true;
    if (S_.fixed) {
      // one inner solve of exactly fixed_iters FP32 steps from zero and its FP64 update:
      // the inner iteration itself, comparable with Algorithm 2 or 3 at that step count
      S_.tol = 0.0;
      S_.inner_tol = 0.0;
      S_.inner_maxit = o.fixed_iters;
      S_.maxit = 1;
    } else {
      if (!(tol > 0)) return HOM_ERR_INVALID;
      S_.tol = tol;
      S_.inner_tol = o.inner_tol > 0 ? o.inner_tol : 1e-4;
      S_.inner_maxit = 10000;
      S_.maxit = o.maxit > 0 ? o.maxit : 50;
    }
    S_.pot = (solver == HOM_CG || solver == HOM_CHEBYSHEV) && o.inner_form == 0 &&
             P->e32.pot_ok();
    return refine_begin(P);
  }

  cudaStream_t st = P->stream;
  cpx<double>* S = (cpx<double>*)P->S;
  Scalars s{};
  for (int a = 0; a < d; ++a) s.E[a] = E[a];
  s.tol = tol;
  s.nE = nE;
  s.maxit = S_.maxit;
  s.fixed = S_.fixed ? 1 : 0;
  s.stop = stop;
  double* x = P->vec[0];
  double* r = P->vec[2];
  double* p = P->vec[3];
  double* q = P->vec[4];
  OpArgs args{};
  if (solver == HOM_RICHARDSON) s.omega = 2.0 / (cA + CA);
  if (solver == HOM_EYRE_MILTON) {
    s.omega = std::sqrt(cA * CA);
    if (P->nc > 3) {  // six-component stiffness: the post-operator reads (C_p + omega I)^{-1}
      int rc0 = shifted_inverse_table(P, s.omega);
      if (rc0) return rc0;
    }
  }
  if (solver == HOM_CHEBYSHEV) {
    s.cheb_c = 0.5 * (CA - cA);
    s.cheb_d = 0.5 * (cA + CA);
    s.alpha = 1.0 / s.cheb_d;
    s.beta = -0.5 * (s.cheb_c / s.cheb_d) * (s.cheb_c / s.cheb_d);
  }
  // the history of the stopping quantity: one entry an iteration (Richardson on the residual:
  // one more, the residual of the last iterate), at most kHistMax kept
  const int hcap = (int)std::min<long long>((long long)S_.maxit + 2, kHistMax);
  if (hcap > P->hist_alloc) {
    if (P->d_hist) cudaFree(P->d_hist);
    P->d_hist = nullptr;
    P->hist_alloc = 0;
    int ar = alloc((void**)&P->d_hist, sizeof(double) * (size_t)hcap);
    if (ar != HOM_OK) return ar;
    P->hist_alloc = hcap;
  }
  s.hist = P->d_hist;
  s.hist_cap = P->hist_alloc;
  int rc = upload_scalars(P, P->d_sc, s);
  if (rc) return rc;
  S_.solver_begun = true;
  HOM_CUDA(cudaEventRecord(P->ev0, st));
  if (solver == HOM_EYRE_MILTON) {
    Ops<double>::fill_const(x, nodes, d, P->d_sc, st);  // x_0 = E
  } else {
    // x_0 = 0; one affine application gives b = -G A E: ||b|| (and r_0 = p_0 = b for CG and
    // Chebyshev, Algorithms 2-3)
    HOM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * len * (solver == HOM_RICHARDSON ? 2 : 1), st));
    HOM_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * len, st));
    Fields<double> f0{};
    f0.xin = x;
    f0.cs = nodes;
    if (solver == HOM_RICHARDSON) {
      f0.out = q;
      P->e64.apply(PRE_AFFINE, PROJ_GAMMA, POST_STORE, f0, S, P->d_sc, args, P->partials,
                   P->counter, 0, st);
    } else {
      f0.out = r;
      f0.p = p;
      P->e64.apply(PRE_AFFINE, PROJ_GAMMA, POST_STORE, f0, S, P->d_sc, args, P->partials,
                   P->counter, 1, st);
    }
    S_.matvecs = 1;
  }
  return check_last();
}

// a session that failed to begin (argument, allocation or CUDA error) is not active
extern "C" int hom_solve_begin(hom_problem* P, const double* E, int solver, double tol,
                               const hom_opts* opts) {
  if (!P || !E) return HOM_ERR_INVALID;
  const int rc = solve_begin_impl(P, E, solver, tol, opts);
  if (rc != HOM_OK) P->sv.active = false;
  return rc;
}

extern "C" int hom_solve_iterate(hom_problem* P, int iterations, int* done) {
  if (!P || !P->sv.active || iterations < 0) return HOM_ERR_INVALID;
  SolveState& S_ = P->sv;
  if (S_.refined) {
    if (!S_.finished)
      for (int k = 0; k < iterations; ++k) refine_enqueue_inner(P);
    int rc = check_last();
    if (rc) return rc;
    if (done) {
      if (!S_.finished) {
        if ((rc = poll(P, P->d_sc2))) return rc;
        if (P->h_sc->done && (rc = refine_outer_update(P))) return rc;
      }
      *done = S_.finished ? 1 : 0;
    }
    return HOM_OK;
  }
  const int cap = S_.maxit + (S_.solver == HOM_RICHARDSON ? 1 : 0);
  for (int k = 0; k < iterations && S_.issued < cap; ++k) enqueue_step(P);
  int rc = check_last();
  if (rc) return rc;
  if (done) {
    if ((rc = poll(P, P->d_sc))) return rc;
    *done = (P->h_sc->done || S_.issued >= cap) ? 1 : 0;
  }
  return HOM_OK;
}

extern "C" int hom_solve_end(hom_problem* P, double* x_dev, double* AH_EE, double* flux,
                             hom_stats* stats) {
  if (!P || !P->sv.active) return HOM_ERR_INVALID;
  SolveState& S_ = P->sv;
  S_.active = false;
  const int d = P->nc;
  const long long nodes = P->nodes;
  const long long len = (long long)d * nodes;
  cudaStream_t st = P->stream;
  int rc;
  if (S_.refined) {
    HOM_CUDA(cudaEventRecord(P->ev1, st));
    HOM_CUDA(cudaEventSynchronize(P->ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, P->ev0, P->ev1);
    double en = 0, fl[kMaxComp] = {};
    if ((rc = energy_eval(P, S_.E, P->vec[0], &en, fl))) return rc;
    if (AH_EE) *AH_EE = en;
    if (flux)
      for (int a = 0; a < d; ++a) flux[a] = fl[a];
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->iterations = S_.outer_it;
      stats->inner_iterations = S_.inner_total;
      stats->matvecs = S_.inner_total + S_.matvecs + S_.outer_it;
      stats->converged = S_.converged ? 1 : 0;
      stats->residual = S_.nb > 0 ? S_.res / S_.nb : 0.0;
      stats->true_residual = stats->residual;  // the outer residual is formed in FP64
      stats->time_ms = ms;
    }
    if (x_dev && (rc = write_corrector(P, P->vec[0], x_dev))) return rc;
    if ((rc = check_last())) return rc;
    if (tma_wait_errors(true) != 0) return HOM_ERR_TIMEOUT;
    return (S_.converged || S_.fixed) ? HOM_OK : HOM_ERR_NOT_CONVERGED;
  }
  rc = poll(P, P->d_sc);
  if (rc) return rc;
  const Scalars fin = *P->h_sc;
  double* result = P->vec[0];
  int matvecs = S_.matvecs + fin.it;
  if (S_.solver == HOM_RICHARDSON) {
    result = P->vec[0] + (fin.result ? len : 0);
    if (fin.converged && S_.stop == HOM_STOP_RESIDUAL) matvecs += 1;
  } else if (S_.solver == HOM_EYRE_MILTON) {
    // e = G x_m (Section 4.4): the conforming part of the non-conforming iterate
    Fields<double> fp{};
    fp.xin = P->vec[0];
    fp.out = P->vec[2];
    fp.cs = nodes;
    OpArgs args{};
    P->e64.apply(PRE_IDENT, PROJ_GAMMA, POST_STORE, fp, (cpx<double>*)P->S, nullptr, args,
                 nullptr, nullptr, 0, st);
    result = P->vec[2];
  }
  HOM_CUDA(cudaEventRecord(P->ev1, st));
  HOM_CUDA(cudaEventSynchronize(P->ev1));
  float ms = 0;
  cudaEventElapsedTime(&ms, P->ev0, P->ev1);
  double en = 0, fl[kMaxComp] = {};
  rc = energy_eval(P, S_.E, result, &en, fl);
  if (rc) return rc;
  if (AH_EE) *AH_EE = en;
  if (flux)
    for (int a = 0; a < d; ++a) flux[a] = fl[a];
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = fin.it;
    stats->matvecs = matvecs;
    stats->converged = fin.converged;
    if (S_.stop == HOM_STOP_INCREMENT)
      stats->residual = fin.last_inc / (S_.nE > 0 ? S_.nE : 1);
    else
      stats->residual = fin.last_res / (fin.nb > 0 ? fin.nb : 1);
    stats->time_ms = ms;
    const double tr = true_residual(P, S_.E, result, P->vec[4]);
    if (S_.solver == HOM_EYRE_MILTON)
      stats->true_residual = tr;  // ||G A (E + e)||, no ||b|| formed by this solver
    else
      stats->true_residual = (fin.nb > 0 && tr >= 0) ? tr / fin.nb : tr;
  }
  if (x_dev && (rc = write_corrector(P, result, x_dev))) return rc;
  if ((rc = check_last())) return rc;
  if (tma_wait_errors(true) != 0) return HOM_ERR_TIMEOUT;
  return (fin.converged || S_.fixed) ? HOM_OK : HOM_ERR_NOT_CONVERGED;
}

extern "C" int hom_solve_history(hom_problem* P, double* out, int cap, int* count) {
  if (!P || cap < 0 || (cap > 0 && !out)) return HOM_ERR_INVALID;
  SolveState& S_ = P->sv;
  int n = 0;
  if (S_.refined) {
    n = (int)S_.outer_hist.size();
    for (int i = 0; i < std::min(n, cap); ++i) out[i] = S_.outer_hist[i];
  } else if (S_.solver_begun) {
    int rc = poll(P, P->d_sc);
    if (rc) return rc;
    n = P->h_sc->nhist;
    const int m = std::min(std::min(n, cap), P->hist_alloc);
    if (m > 0) {
      HOM_CUDA(cudaMemcpyAsync(out, P->d_hist, sizeof(double) * (size_t)m,
                               cudaMemcpyDeviceToHost, P->stream));
      HOM_CUDA(cudaStreamSynchronize(P->stream));
    }
  }
  if (count) *count = n;
  return check_last();
}

extern "C" int hom_solve_current(hom_problem* P, double* x_dev) {
  if (!P || !x_dev || !P->sv.active) return HOM_ERR_INVALID;
  SolveState& S_ = P->sv;
  const long long nodes = P->nodes;
  const long long len = (long long)P->nc * nodes;
  cudaStream_t st = P->stream;
  const double* cur = P->vec[0];
  if (!S_.refined) {
    int rc = poll(P, P->d_sc);
    if (rc) return rc;
    if (S_.solver == HOM_RICHARDSON) cur = P->vec[0] + (P->h_sc->result ? len : 0);
    if (S_.solver == HOM_EYRE_MILTON) {
      // e = G x_m (Section 4.4), as the end of the solve returns it, into the free vector
      Fields<double> fp{};
      fp.xin = P->vec[0];
      fp.out = P->vec[4];
      fp.cs = nodes;
      OpArgs args{};
      P->e64.apply(PRE_IDENT, PROJ_GAMMA, POST_STORE, fp, (cpx<double>*)P->S, nullptr, args,
                   nullptr, nullptr, 0, st);
      cur = P->vec[4];
    }
  }
  (void)len;
  return write_corrector(P, cur, x_dev);
}

extern "C" int hom_solve_nonconformity(hom_problem* P, double* value) {
  if (!P || !value || !P->sv.active) return HOM_ERR_INVALID;
  SolveState& S_ = P->sv;
  const long long nodes = P->nodes;
  const long long len = (long long)P->nc * nodes;
  cudaStream_t st = P->stream;
  const double* cur = P->vec[0];
  Scalars s{};  // E for the Eyre-Milton iterate, zero for the conforming solvers
  int rc;
  if (!S_.refined) {
    if ((rc = poll(P, P->d_sc))) return rc;
    if (S_.solver == HOM_RICHARDSON) cur = P->vec[0] + (P->h_sc->result ? len : 0);
    if (S_.solver == HOM_EYRE_MILTON)
      for (int a = 0; a < P->nc; ++a) s.E[a] = S_.E[a];
  }
  // G x into the solver's free vector (no solver keeps state there between steps)
  double* g = P->vec[4];
  Fields<double> f{};
  f.xin = cur;
  f.out = g;
  f.cs = nodes;
  OpArgs args{};
  P->e64.apply(PRE_IDENT, PROJ_GAMMA, POST_STORE, f, (cpx<double>*)P->S, nullptr, args, nullptr,
               nullptr, 0, st);
  if ((rc = upload_scalars(P, P->d_aux, s))) return rc;
  k_nonconf<double><<<P->red_grid, kThreads, 0, st>>>(g, cur, P->nc, nodes, P->partials,
                                                       P->counter, P->d_aux);
  if ((rc = check_last()) || (rc = poll(P, P->d_aux))) return rc;
  *value = P->h_sc->last_res;
  return HOM_OK;
}

// ---------------------------------------------------------------------------------------
// snapshot / restore of an FP64 session: the five solver vectors, the device scalars, the
// stored history and the host-side counters behind a header that identifies the session
// ---------------------------------------------------------------------------------------
namespace {

struct SnapHeader {
  unsigned magic;
  int nc, M[3];
  long long nodes;
  int integration, solver, stop, fixed, maxit;
  int issued, matvecs;
  double E[kMaxComp], nE;
  Scalars sc;            // the device scalars at the snapshot (hist is the source's pointer)
  long long nhist_kept;  // history entries that follow the vectors
};
constexpr unsigned kSnapMagic = 0x686f6d53u;  // "homS"

size_t snap_vec_bytes(const hom_problem* P) {
  return sizeof(double) * 5 * (size_t)P->nc * (size_t)P->nodes;
}

// the size a snapshot of P's session takes: header, vectors, room for the whole history
size_t snap_bytes(const hom_problem* P) {
  return sizeof(SnapHeader) + snap_vec_bytes(P) + sizeof(double) * (size_t)P->hist_alloc;
}

bool snap_ok(const hom_problem* P) {
  return P && P->sv.active && !P->sv.refined && P->sv.solver_begun;
}

}  // namespace

extern "C" int hom_solve_snapshot_size(hom_problem* P, size_t* bytes) {
  if (!P || !bytes || !P->sv.active) return HOM_ERR_INVALID;
  if (P->sv.refined) return HOM_ERR_UNSUPPORTED;
  if (!snap_ok(P)) return HOM_ERR_INVALID;
  *bytes = snap_bytes(P);
  return HOM_OK;
}

extern "C" int hom_solve_snapshot(hom_problem* P, void* host_buf, size_t bytes) {
  if (!P || !host_buf || !P->sv.active) return HOM_ERR_INVALID;
  if (P->sv.refined) return HOM_ERR_UNSUPPORTED;
  if (!snap_ok(P) || bytes < snap_bytes(P)) return HOM_ERR_INVALID;
  const SolveState& S_ = P->sv;
  HOM_CUDA(cudaStreamSynchronize(P->stream));
  SnapHeader h{};
  h.magic = kSnapMagic;
  h.nc = P->nc;
  for (int a = 0; a < 3; ++a) h.M[a] = P->M[a];
  h.nodes = P->nodes;
  h.integration = P->integration;
  h.solver = S_.solver;
  h.stop = S_.stop;
  h.fixed = S_.fixed ? 1 : 0;
  h.maxit = S_.maxit;
  h.issued = S_.issued;
  h.matvecs = S_.matvecs;
  for (int a = 0; a < kMaxComp; ++a) h.E[a] = S_.E[a];
  h.nE = S_.nE;
  int rc = poll(P, P->d_sc);
  if (rc) return rc;
  h.sc = *P->h_sc;
  h.nhist_kept = (h.sc.hist != nullptr) ? std::min<long long>(h.sc.nhist, h.sc.hist_cap) : 0;
  unsigned char* out = static_cast<unsigned char*>(host_buf);
  std::memcpy(out, &h, sizeof(h));
  cudaStream_t st = P->stream;
  HOM_CUDA(cudaMemcpyAsync(out + sizeof(h), P->vbase, snap_vec_bytes(P), cudaMemcpyDeviceToHost,
                           st));
  if (h.nhist_kept > 0)
    HOM_CUDA(cudaMemcpyAsync(out + sizeof(h) + snap_vec_bytes(P), h.sc.hist,
                             sizeof(double) * (size_t)h.nhist_kept, cudaMemcpyDeviceToHost, st));
  HOM_CUDA(cudaStreamSynchronize(st));
  return check_last();
}

extern "C" int hom_solve_restore(hom_problem* P, const void* host_buf, size_t bytes) {
  if (!P || !host_buf || !P->sv.active) return HOM_ERR_INVALID;
  if (P->sv.refined) return HOM_ERR_UNSUPPORTED;
  if (!snap_ok(P) || bytes < sizeof(SnapHeader)) return HOM_ERR_INVALID;
  SnapHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  SolveState& S_ = P->sv;
  // the same shape, solver, stopping rule, limits and macroscopic field as the session begun
  // here; the coefficients and the launch plan are the caller's to keep equal
  bool same = h.magic == kSnapMagic && h.nc == P->nc && h.nodes == P->nodes &&
              h.integration == P->integration && h.solver == S_.solver && h.stop == S_.stop &&
              h.fixed == (S_.fixed ? 1 : 0) && h.maxit == S_.maxit && h.nE == S_.nE &&
              h.nhist_kept >= 0 &&
              bytes >= sizeof(h) + snap_vec_bytes(P) + sizeof(double) * (size_t)h.nhist_kept;
  for (int a = 0; a < 3; ++a) same = same && h.M[a] == P->M[a];
  for (int a = 0; a < kMaxComp; ++a) same = same && h.E[a] == S_.E[a];
  if (!same) return HOM_ERR_INVALID;
  cudaStream_t st = P->stream;
  int rc = poll(P, P->d_sc);  // also waits for the steps already enqueued
  if (rc) return rc;
  Scalars sc = h.sc;
  sc.hist = P->h_sc->hist;  // this session's history buffer and capacity
  sc.hist_cap = P->h_sc->hist_cap;
  const unsigned char* in = static_cast<const unsigned char*>(host_buf);
  HOM_CUDA(cudaMemcpyAsync(P->vbase, in + sizeof(h), snap_vec_bytes(P), cudaMemcpyHostToDevice,
                           st));
  const long long keep = sc.hist ? std::min<long long>(h.nhist_kept, sc.hist_cap) : 0;
  if (keep > 0)
    HOM_CUDA(cudaMemcpyAsync(sc.hist, in + sizeof(h) + snap_vec_bytes(P),
                             sizeof(double) * (size_t)keep, cudaMemcpyHostToDevice, st));
  if ((rc = upload_scalars(P, P->d_sc, sc))) return rc;  // synchronises the stream
  // the polling interval and output flags stay those this session was begun with
  S_.issued = h.issued;
  S_.matvecs = h.matvecs;
  return check_last();
}

extern "C" int hom_solve(hom_problem* P, const double* E, int solver, double tol,
                         const hom_opts* opts, double* x_dev, double* AH_EE, double* flux,
                         hom_stats* stats) {
  int rc = hom_solve_begin(P, E, solver, tol, opts);
  if (rc) return rc;
  int done = 0;
  while (!done) {
    rc = hom_solve_iterate(P, P->sv.check, &done);
    if (rc) return rc;
  }
  return hom_solve_end(P, x_dev, AH_EE, flux, stats);
}

extern "C" int hom_energy(hom_problem* P, const double* E, const double* x_dev, double* energy,
                          double* flux) {
  if (!P || !E) return HOM_ERR_INVALID;
  return energy_eval(P, E, x_dev, energy, flux);
}

extern "C" int hom_prolongate(hom_problem* Cp, hom_problem* Fp, const double* x_dev,
                              double* y_dev) {
  if (!Cp || !Fp || !x_dev || !y_dev || Cp->d != Fp->d) return HOM_ERR_INVALID;
  if (Cp->nc != Cp->d || Fp->nc != Fp->d) return HOM_ERR_UNSUPPORTED;  // strain fields
  const int d = Cp->d;
  for (int a = 0; a < d; ++a)
    if (Fp->M[a] < Cp->M[a]) return HOM_ERR_INVALID;
  cudaStream_t st = Cp->stream;
  // F_N on the coarse grid (unscaled), then 1/|N| and the zero padding into Z_M, then F_M^{-1}
  Cp->e64.forward(x_dev, (cpx<double>*)Cp->S, d, st);
  HOM_CUDA(cudaMemsetAsync(Fp->S, 0, Fp->S_bytes, st));
  const PassGeom& gn = Cp->e64.g;
  const PassGeom& gm = Fp->e64.g;
  const int n1 = d == 3 ? gn.n[1] : 1, m1 = d == 3 ? gm.n[1] : 1;
  Ops<double>::pad_spectrum((const cpx<double>*)Cp->S, (cpx<double>*)Fp->S, d, gn.n[0], n1,
                            gn.nh, gm.n[0], m1, gm.nh, 1.0 / (double)gn.nodes, gn.scs, gm.scs, st);
  if (Fp->stream != st) {
    HOM_CUDA(cudaStreamSynchronize(st));
  }
  Fp->e64.inverse((cpx<double>*)Fp->S, y_dev, d, Fp->stream);
  return check_last();
}

extern "C" int hom_restrict(hom_problem* P, const double* x_dev, double* y_dev) {
  if (!P || !x_dev || !y_dev) return HOM_ERR_INVALID;
  return restrict_field(P, x_dev, y_dev);
}

extern "C" int hom_bound(hom_problem* gani, hom_problem* ga, const double* E,
                         const double* x_dev, double* UE) {
  if (!gani || !ga || !E || !x_dev || !UE) return HOM_ERR_INVALID;
  if (gani->integration != HOM_APPROX || ga->integration != HOM_EXACT || gani->d != ga->d)
    return HOM_ERR_INVALID;
  if (gani->nc != gani->d) return HOM_ERR_UNSUPPORTED;  // strain fields (no exact integration)
  for (int a = 0; a < gani->d; ++a)
    if (ga->N[a] != gani->N[a]) return HOM_ERR_INVALID;
  double* y = ga->vec[4];
  int rc = hom_prolongate(gani, ga, x_dev, y);
  if (rc) return rc;
  HOM_CUDA(cudaStreamSynchronize(ga->stream));
  return energy_eval(ga, E, y, UE, nullptr);
}

// ---------------------------------------------------------------------------------------
// autotuner: time candidate launch plans of P's grid and keep the fastest
// ---------------------------------------------------------------------------------------
namespace {

template <typename T>
int tune_engine(hom_problem* P, Engine<T>& E, T* x, T* y, int reps, const std::vector<int>& rmaxes,
                const std::vector<size_t>& budgets, PlanChoice* best, double* best_ms) {
  const int d = P->d;
  const size_t cap = (size_t)dynamic_smem_cap();
  double best_t = 1e300;
  PlanChoice choice{E.rmax_used, E.budget_used, E.threads_used, E.two_line};
  // FP32: plans on which the inner solves can run in potential coordinates (specialised plans
  // on every axis) win over any other, since the timed operator is not the step those solves
  // run; among them, and among the rest, the fastest operator wins
  bool best_pot = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Fields<T> f{};
  f.xin = x;
  f.out = y;
  f.cs = P->nodes;
  OpArgs args{};
  for (int rmax : rmaxes)
    for (size_t budget : budgets)
      for (int threads : {kThreads / 2, kThreads})
        for (bool two : {true, false}) {
      if (budget > cap) continue;
      E.release_plan();
      if (E.init(d, P->M, P->N, budget, rmax, threads, two, P->nc) != HOM_OK) continue;
      if (!two && !Ops<T>::two_line_ok(E.g, E.plan[0], E.plan[1])) continue;  // same plan
      E.apply(PRE_LINEAR, PROJ_GAMMA, POST_STORE, f, (cpx<T>*)P->S, nullptr, args, nullptr,
              nullptr, 0, P->stream);  // warm-up
      cudaEventRecord(e0, P->stream);
      for (int r = 0; r < reps; ++r)
        E.apply(PRE_LINEAR, PROJ_GAMMA, POST_STORE, f, (cpx<T>*)P->S, nullptr, args, nullptr,
                nullptr, 0, P->stream);
      cudaEventRecord(e1, P->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return check_last();
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const bool pot = E.pot_ok();
      if ((pot && !best_pot) || (pot == best_pot && ms < best_t)) {
        best_t = ms;
        best_pot = pot;
        choice = PlanChoice{rmax, budget, threads, E.two_line};
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  E.release_plan();
  const int rc = E.init(d, P->M, P->N, choice.budget, choice.rmax, choice.threads,
                        choice.two_line, P->nc);
  *best = choice;
  *best_ms = best_t / reps;
  return rc ? rc : check_last();
}

}  // namespace

extern "C" int hom_set_plan(hom_problem* P, const hom_tune_report* plan) {
  if (!P || !plan || P->sv.active) return HOM_ERR_INVALID;
  const size_t cap = (size_t)dynamic_smem_cap();
  auto ok = [&](int rmax, int kb, int threads) {
    return rmax >= 3 && rmax <= kMaxRadix && kb > 0 && (size_t)kb * 1024 <= cap &&
           (threads == kThreads / 2 || threads == kThreads);
  };
  if (!ok(plan->rmax64, plan->smem_kb64, plan->threads64)) return HOM_ERR_INVALID;
  const bool f32 = P->precision == HOM_FP32_REFINED;
  if (f32 && !ok(plan->rmax32, plan->smem_kb32, plan->threads32)) return HOM_ERR_INVALID;
  P->e64.release_plan();
  int rc = P->e64.init(P->d, P->M, P->N, (size_t)plan->smem_kb64 * 1024, plan->rmax64,
                       plan->threads64, true, P->nc);
  if (rc) return rc;
  if (f32) {
    P->e32.release_plan();
    rc = P->e32.init(P->d, P->M, P->N, (size_t)plan->smem_kb32 * 1024, plan->rmax32,
                     plan->threads32, plan->two_line32 != 0, P->nc);
    if (rc) return rc;
  }
  return check_last();
}

extern "C" int hom_autotune(hom_problem* P, int reps, hom_tune_report* report) {
  if (!P || P->sv.active) return HOM_ERR_INVALID;
  if (reps < 1) reps = 3;
  hom_tune_report rep{};
  PlanChoice c{};
  double ms = 0;
  const std::vector<size_t> budgets = {56 * 1024, 80 * 1024, 96 * 1024, 110 * 1024, 150 * 1024,
                                       200 * 1024};
  int rc = tune_engine<double>(P, P->e64, P->vec[0], P->vec[1], reps, {9, 15}, budgets, &c, &ms);
  if (rc) return rc;
  rep.rmax64 = c.rmax;
  rep.smem_kb64 = (int)(c.budget / 1024);
  rep.threads64 = c.threads;
  rep.ms64 = ms;
  {
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_table()[tune_key(8, P->d, P->M, P->N, P->nc)] = c;
  }
  if (P->precision == HOM_FP32_REFINED) {
    rc = tune_engine<float>(P, P->e32, P->fvec[0], P->fvec[1], reps, {9, 15, 27}, budgets, &c, &ms);
    if (rc) return rc;
    rep.rmax32 = c.rmax;
    rep.smem_kb32 = (int)(c.budget / 1024);
    rep.threads32 = c.threads;
    rep.two_line32 = c.two_line ? 1 : 0;
    rep.ms32 = ms;
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_table()[tune_key(4, P->d, P->M, P->N, P->nc)] = c;
  }
  if (report) *report = rep;
  return HOM_OK;
}
