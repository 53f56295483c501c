// hom_apply_static: one operator application that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns every byte of device
// memory through its own allocator or a fixed budget, a plugin loaded into such an
// application, or a latency-critical loop that must not pay for cudaMalloc/cudaFree (both can
// synchronise the whole device and stall unrelated streams). For them this file keeps the
// work memory of the operator (half spectrum, twiddle tables, coefficient table) in one
// file-scope __device__ array of HOM_STATIC_SCRATCH_BYTES, which every GPU that loads the
// library holds until the process exits. The caller passes inputs and outputs only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hom.h"
#include "ops.h"
#include "passes.cuh"

using namespace hom;

namespace {

constexpr size_t kTwBytes = 64 * 1024;                 // three twiddle tables (<= 1023 each)
constexpr size_t kTabBytes = 512 * 1024;               // coefficient table (<= 65536 doubles)
constexpr size_t kSpecOff = kTwBytes + kTabBytes;      // half spectrum after both
static_assert(3 * kMaxAxis * sizeof(cpx<double>) <= kTwBytes, "twiddle region too small");

}  // namespace

// The scratch itself. Host code must not use this name as an address: it is a host-side
// stand-in for the device symbol. The device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_hom_scratch[HOM_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_base[kMaxDevices] = {};

// Per-device set-up, once, with that device current: resolve the scratch address, upload the
// DFT constants and raise the kernels' shared-memory limits. No allocation.
int static_setup(int dev, unsigned char** base) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (g_static_base[dev] != nullptr) {
    *base = g_static_base[dev];
    return HOM_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_hom_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return HOM_ERR_CUDA;
  }
  if (Ops<double>::upload_constants() != cudaSuccess || Ops<double>::prepare(3) != cudaSuccess) {
    cudaGetLastError();
    return HOM_ERR_CUDA;
  }
  g_static_base[dev] = static_cast<unsigned char*>(p);
  *base = g_static_base[dev];
  return HOM_OK;
}

// radix plan of one axis: prime factors (<= 31) grouped first-fit into register radices <= 15
bool plan_static_axis(int n, AxisPlan* P) {
  if (n < 3 || n > kMaxAxis || n % 2 == 0) return false;
  int groups[kMaxStages];
  int ng = 0, rem = n;
  for (int R : {31, 29, 23, 19, 17, 13, 11, 7, 5, 3})
    while (rem % R == 0) {
      rem /= R;
      int best = -1;
      for (int gi = 0; gi < ng; ++gi)
        if (groups[gi] * R <= 15 && (best < 0 || groups[gi] > groups[best])) best = gi;
      if (best >= 0) {
        groups[best] *= R;
      } else {
        if (ng >= kMaxStages) return false;
        groups[ng++] = R;
      }
    }
  if (rem != 1) return false;
  std::sort(groups, groups + ng, [](int a, int b) { return a > b; });
  P->n = n;
  P->nst = ng;
  int p = 1;
  for (int s = 0; s < kMaxStages; ++s) {
    P->pprev[s] = s < ng ? p : 0;
    P->radix[s] = s < ng ? groups[s] : 0;
    if (s < ng) p *= groups[s];
  }
  plan_fastdivs(P);
  return true;
}

// extreme eigenvalues of a symmetric d x d tensor (d <= 3) by Jacobi rotations; false unless SPD
bool static_spd(const double* t, int d, double* lo, double* hi) {
  double a[3][3];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) a[i][j] = t[i * d + j];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(a[i][j] - a[j][i]) > 1e-12 * (std::fabs(a[i][j]) + std::fabs(a[j][i]) + 1e-300))
        return false;
  for (int sweep = 0; sweep < 50; ++sweep)
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
  *lo = *hi = a[0][0];
  for (int i = 1; i < d; ++i) {
    *lo = std::min(*lo, a[i][i]);
    *hi = std::max(*hi, a[i][i]);
  }
  return *lo > 0;
}

}  // namespace

extern "C" int hom_apply_static(int d, const int* N, const void* phase_dev, int index_bytes,
                                const double* table, int nphase, int op, const double* E,
                                const double* x_dev, double* y_dev, void* stream) {
  if ((d != 2 && d != 3) || !N || !phase_dev || !table || !x_dev || !y_dev) return HOM_ERR_INVALID;
  if (index_bytes != 1 && index_bytes != 2) return HOM_ERR_INVALID;
  if (nphase < 1 || (index_bytes == 1 && nphase > 256)) return HOM_ERR_INVALID;
  if (op < HOM_OP_AFFINE || op > HOM_OP_EM || (op == HOM_OP_AFFINE && !E)) return HOM_ERR_INVALID;
  PassGeom g{};
  AxisPlan plan[3]{};
  g.D = d;
  g.nodes = 1;
  for (int a = 0; a < d; ++a) {
    if (!plan_static_axis(N[a], &plan[a])) return HOM_ERR_INVALID;
    g.n[a] = N[a];
    g.nodes *= N[a];
  }
  for (int a = d; a < 3; ++a) g.n[a] = 1;
  const int nl = N[d - 1];
  g.nh = (nl + 1) / 2;
  g.nlines = g.nodes / nl;
  g.scs = g.nlines * g.nh;

  // ---- size limits of the static scratch ----
  const size_t spec_bytes = sizeof(cpx<double>) * (size_t)d * (size_t)g.scs;
  const bool iso_table = [&] {
    for (int p = 0; p < nphase; ++p)
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          const double v = table[(size_t)p * d * d + i * d + j];
          if ((i != j && v != 0.0) || (i == j && v != table[(size_t)p * d * d])) return false;
        }
    return true;
  }();
  const size_t tab_bytes = sizeof(double) * (size_t)nphase * (iso_table ? 1 : d * d);
  if (kSpecOff + spec_bytes > (size_t)HOM_STATIC_SCRATCH_BYTES || tab_bytes > kTabBytes)
    return HOM_ERR_SCRATCH;

  // ---- coefficients: SPD phases and the bounds c_A, C_A (eq. (A)) ----
  double cA = 1e300, CA = -1e300;
  std::vector<double> tab;
  for (int p = 0; p < nphase; ++p) {
    double lo, hi;
    if (!static_spd(table + (size_t)p * d * d, d, &lo, &hi)) return HOM_ERR_INVALID;
    cA = std::min(cA, lo);
    CA = std::max(CA, hi);
    if (iso_table) tab.push_back(table[(size_t)p * d * d]);
  }
  if (!iso_table) tab.assign(table, table + (size_t)nphase * d * d);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HOM_ERR_CUDA;
  unsigned char* base = nullptr;
  int rc = static_setup(dev, &base);
  if (rc != HOM_OK) return rc;

  // ---- launch geometry (the default budget of hom_create) ----
  if (!Ops<double>::plan_geometry(d, N, plan, 110 * 1024, kThreads, &g))
    return HOM_ERR_UNSUPPORTED;

  // ---- twiddles and table into the scratch (ordered on the caller's stream) ----
  cudaStream_t st = (cudaStream_t)stream;
  cpx<double>* tw[3] = {nullptr, nullptr, nullptr};
  std::vector<cpx<double>> tw_h((size_t)3 * kMaxAxis);
  const long double twopi = 6.283185307179586476925286766559005768L;
  for (int a = 0; a < d; ++a) {
    tw[a] = reinterpret_cast<cpx<double>*>(base) + (size_t)a * kMaxAxis;
    for (int j = 0; j < N[a]; ++j) {
      const long double t = -twopi * (long double)j / (long double)N[a];
      tw_h[(size_t)a * kMaxAxis + j].x = (double)cosl(t);
      tw_h[(size_t)a * kMaxAxis + j].y = (double)sinl(t);
    }
  }
  double* tab_dev = reinterpret_cast<double*>(base + kTwBytes);
  cpx<double>* S = reinterpret_cast<cpx<double>*>(base + kSpecOff);
  if (cudaMemcpyAsync(base, tw_h.data(), sizeof(cpx<double>) * 3 * kMaxAxis,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(tab_dev, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice,
                      st) != cudaSuccess) {
    cudaGetLastError();
    return HOM_ERR_CUDA;
  }

  // ---- one application: the same passes as hom_apply ----
  MatView<double> mat{};
  mat.kind = iso_table ? MAT_PHASE_ISO : MAT_PHASE_TENSOR;
  mat.ph8 = index_bytes == 1 ? static_cast<const uint8_t*>(phase_dev) : nullptr;
  mat.ph16 = index_bytes == 2 ? static_cast<const uint16_t*>(phase_dev) : nullptr;
  mat.table = tab_dev;
  ProjGeom pg{};
  pg.C = g.scs / N[0];
  pg.cs = g.scs;
  pg.n1 = d == 3 ? N[1] : 1;
  pg.nh = g.nh;
  pg.fdnh = make_fastdiv(g.nh);
  for (int a = 0; a < 3; ++a) pg.hw[a] = a < d ? (N[a] - 1) / 2 : 0;
  pg.scale = 1.0 / (double)g.nodes;
  OpArgs args{};
  for (int a = 0; a < d; ++a) args.E[a] = E ? E[a] : 0.0;
  args.omega = std::sqrt(cA * CA);
  Fields<double> f{};
  f.xin = x_dev;
  f.out = y_dev;
  f.cs = g.nodes;
  const int pre = op == HOM_OP_AFFINE ? PRE_AFFINE : op == HOM_OP_LINEAR ? PRE_LINEAR
                : op == HOM_OP_PROJECT ? PRE_IDENT : PRE_EM;
  const int mode = op == HOM_OP_EM ? PROJ_EM : PROJ_GAMMA;
  Ops<double>::line_fwd(g, pre, f, S, plan[d - 1], tw[d - 1], d, mat, nullptr, args, st);
  if (d == 3) Ops<double>::strided(g, 1, 0, S, plan[1], tw[1], d, nullptr, st);
  Ops<double>::proj(g, mode, S, plan[0], tw[0], pg, nullptr, st);
  if (d == 3) Ops<double>::strided(g, 1, 1, S, plan[1], tw[1], d, nullptr, st);
  Ops<double>::line_inv(g, POST_STORE, S, f, plan[d - 1], tw[d - 1], d, mat, nullptr, args,
                        nullptr, nullptr, 0, st);
  if (cudaGetLastError() != cudaSuccess) return HOM_ERR_CUDA;
  return HOM_OK;
}
