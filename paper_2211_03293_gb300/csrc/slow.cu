// Slow partition and the MRI step driver: periodic central advection-diffusion
// f^S, the stage forcing of the MIS form, and one explicit MRI (Knoth-Wolke
// "MRI3") slow step built from them and mri_stage_fast.
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace mri {

constexpr int kMaxTaps = 13;   // 4th order in 3-D: 4 neighbours per axis plus the centre

struct Stencil {
  int nx, ny, nz, n, ntap;
  int axis[kMaxTaps], off[kMaxTaps];
  double w[kMaxTaps];
};

// One thread per (cell, component): f^S = sum over taps of w_tap * y[neighbour].  The
// taps fold advection and diffusion of every axis into one weight per neighbour.
__global__ void slow_rhs_kernel(const double* __restrict__ y, double* __restrict__ f, Stencil s) {
  const long long total = (long long)s.nx * s.ny * s.nz * s.n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cell = e / s.n;
    const int q = (int)(e - cell * s.n);
    const int i = (int)(cell % s.nx);
    const int j = (int)((cell / s.nx) % s.ny);
    const int k = (int)(cell / ((long long)s.nx * s.ny));
    double acc = 0.0;
#pragma unroll 1
    for (int t = 0; t < s.ntap; ++t) {
      int ii = i, jj = j, kk = k;
      if (s.axis[t] == 0) { ii += s.off[t]; ii += (ii < 0) ? s.nx : 0; ii -= (ii >= s.nx) ? s.nx : 0; }
      else if (s.axis[t] == 1) { jj += s.off[t]; jj += (jj < 0) ? s.ny : 0; jj -= (jj >= s.ny) ? s.ny : 0; }
      else { kk += s.off[t]; kk += (kk < 0) ? s.nz : 0; kk -= (kk >= s.nz) ? s.nz : 0; }
      const long long nb = ((long long)kk * s.ny + jj) * s.nx + ii;
      acc = fma(s.w[t], __ldg(y + nb * s.n + q), acc);
    }
    f[e] = acc;
  }
}

// phi = sum_{j < m} G_j fS_j elementwise.
__global__ void combine_kernel(double* __restrict__ phi, const double* __restrict__ fS, long long len, int m,
                               double g0, double g1, double g2) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double v = g0 * fS[e];
    if (m > 1) v = fma(g1, fS[len + e], v);
    if (m > 2) v = fma(g2, fS[2 * len + e], v);
    phi[e] = v;
  }
}

static bool grid_ok(const mri_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->dx > 0 && std::isfinite(g->dx) &&
         (g->order == 2 || g->order == 4) && std::isfinite(g->u[0]) && std::isfinite(g->u[1]) &&
         std::isfinite(g->u[2]) && g->D >= 0 && std::isfinite(g->D) &&
         (long long)g->nx * g->ny * g->nz <= (1ll << 31) - 1;
}

// Tap weights.  2nd order: d1 = (f+ - f-)/(2dx), d2 = (f+ - 2f + f-)/dx^2.  4th order:
// d1 = (-f++ + 8f+ - 8f- + f--)/(12dx), d2 = (-f++ + 16f+ - 30f + 16f- - f--)/(12dx^2).
// f^S = sum_axes (-u_a d1 + D d2).
static Stencil make_stencil(const mri_grid* g, int n) {
  Stencil s{};
  s.nx = g->nx; s.ny = g->ny; s.nz = g->nz; s.n = n;
  const int N[3] = {g->nx, g->ny, g->nz};
  const double dx = g->dx, D = g->D;
  double centre = 0.0;
  int t = 1;
  for (int a = 0; a < 3; ++a) {
    if (N[a] == 1) continue;
    const double u = g->u[a];
    if (g->order == 2) {
      const double c1 = u / (2.0 * dx), c2 = D / (dx * dx);
      s.axis[t] = a; s.off[t] = 1; s.w[t] = -c1 + c2; ++t;
      s.axis[t] = a; s.off[t] = -1; s.w[t] = c1 + c2; ++t;
      centre += -2.0 * c2;
    } else {
      const double c1 = u / (12.0 * dx), c2 = D / (12.0 * dx * dx);
      s.axis[t] = a; s.off[t] = 1; s.w[t] = -8.0 * c1 + 16.0 * c2; ++t;
      s.axis[t] = a; s.off[t] = -1; s.w[t] = 8.0 * c1 + 16.0 * c2; ++t;
      s.axis[t] = a; s.off[t] = 2; s.w[t] = c1 - c2; ++t;
      s.axis[t] = a; s.off[t] = -2; s.w[t] = -c1 - c2; ++t;
      centre += -30.0 * c2;
    }
  }
  s.axis[0] = 0; s.off[0] = 0; s.w[0] = centre;
  s.ntap = t;
  return s;
}

static int launch_slow(const double* y, double* f, int n, const mri_grid* g, cudaStream_t st) {
  Stencil s = make_stencil(g, n);
  const long long total = (long long)g->nx * g->ny * g->nz * n;
  if (total == 0) return MRI_OK;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  const long long cap = (long long)device_sm_count() * 16;
  if (blocks > cap) blocks = cap;
  slow_rhs_kernel<<<(int)blocks, threads, 0, st>>>(y, f, s);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

// Knoth-Wolke third-order explicit RK in MIS form: c = (0, 1/3, 3/4, 1), rows
// a_2 = (1/3), a_3 = (-3/16, 15/16), a_4 = b = (1/6, 3/10, 8/15).  Stage i's constant
// forcing is sum_j G_ij fS_j with G_ij = (a_ij - a_{i-1,j}) / (c_i - c_{i-1}).
struct Kw3 {
  double c[4];
  double G[4][3];
};

static Kw3 kw3_coupling() {
  const double A[4][3] = {{0.0, 0.0, 0.0},
                          {1.0 / 3.0, 0.0, 0.0},
                          {-3.0 / 16.0, 15.0 / 16.0, 0.0},
                          {1.0 / 6.0, 3.0 / 10.0, 8.0 / 15.0}};
  Kw3 k{};
  k.c[0] = 0.0; k.c[1] = 1.0 / 3.0; k.c[2] = 3.0 / 4.0; k.c[3] = 1.0;
  for (int i = 1; i < 4; ++i)
    for (int j = 0; j < 3; ++j) k.G[i][j] = (A[i][j] - A[i - 1][j]) / (k.c[i] - k.c[i - 1]);
  return k;
}

}  // namespace mri

extern "C" int mri_slow_rhs(const double* y, double* fS, int n, const mri_grid* grid, double t, void* stream) {
  (void)t;
  if (!mri::grid_ok(grid) || n < 1 || !y || !fS) return MRI_EINVAL;
  return mri::launch_slow(y, fS, n, grid, static_cast<cudaStream_t>(stream));
}

extern "C" int mri_stage_forcing(const double* fS, int nslow, long long len, const double* coeffs, double* phi,
                                 void* stream) {
  if (nslow < 1 || nslow > 3 || len < 0 || !coeffs || (len > 0 && (!fS || !phi))) return MRI_EINVAL;
  for (int j = 0; j < nslow; ++j)
    if (!std::isfinite(coeffs[j])) return MRI_EINVAL;
  if (len == 0) return MRI_OK;
  const int threads = 256;
  long long blocks = (len + threads - 1) / threads;
  const long long cap = (long long)mri::device_sm_count() * 16;
  if (blocks > cap) blocks = cap;
  mri::combine_kernel<<<(int)blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
      phi, fS, len, nslow, coeffs[0], nslow > 1 ? coeffs[1] : 0.0, nslow > 2 ? coeffs[2] : 0.0);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_method_coupling(int mri_method, double* c, double* G, int* nstages) {
  if (mri_method != MRI_KW3 || !c || !G || !nstages) return MRI_EINVAL;
  const mri::Kw3 k = mri::kw3_coupling();
  *nstages = 4;
  for (int i = 0; i < 4; ++i) {
    c[i] = k.c[i];
    for (int j = 0; j < 3; ++j) G[i * 3 + j] = (i == 0) ? 0.0 : k.G[i][j];
  }
  return MRI_OK;
}

extern "C" size_t mri_step_workspace_size(const mri_grid* grid, int n) {
  if (!mri::grid_ok(grid) || n < 1) return 0;
  const size_t len = (size_t)grid->nx * grid->ny * grid->nz * n;
  return 4 * len * sizeof(double);   // three f^S evaluations and the stage forcing
}

using mri::mri_stage_fast_checked;

namespace mri {
namespace {

// The host-side checks of an MRI step's arguments, workspace aside: MRI_OK, MRI_EINVAL
// (bad argument, or a mechanism loaded on another device) or MRI_ECUDA.
int step_args_check(const double* y, const double* p, const mri_grid* grid, double H, double h, int mri_method,
                    const mri_mech* mech, const mri_fast_opts* opts) {
  if (!grid_ok(grid) || !mech || !opts || !y || !p || mri_method != MRI_KW3) return MRI_EINVAL;
  if (!(H > 0) || !(h > 0) || !std::isfinite(H) || !std::isfinite(h)) return MRI_EINVAL;
  if (!fast_opts_ok(opts) || opts->time_budget_s != 0.0) return MRI_EINVAL;
  return mech_device_check(*reinterpret_cast<const Mech*>(mech));
}

}  // namespace
}  // namespace mri

extern "C" int mri_step(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
                        int mri_method, const mri_mech* mech, const mri_fast_opts* opts, void* workspace,
                        size_t workspace_bytes, int32_t* cell_status, int32_t* cell_stats, int32_t* n_failed,
                        void* stream) {
  (void)t;
  if (const int rc = mri::step_args_check(y, p, grid, H, h, mri_method, mech, opts)) return rc;
  const mri::Mech* m = reinterpret_cast<const mri::Mech*>(mech);
  const int n = m->L.n;
  const size_t need = mri_step_workspace_size(grid, n);
  if (!workspace || workspace_bytes < need) return MRI_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ncell = grid->nx * grid->ny * grid->nz;
  const long long len = (long long)ncell * n;
  double* fS = static_cast<double*>(workspace);
  double* phi = fS + 3 * len;
  const mri::Kw3 k = mri::kw3_coupling();
  // per-cell status is sticky over the three stages: cleared here, set by a failing stage
  if (cell_status && cudaMemsetAsync(cell_status, 0, sizeof(int32_t) * (size_t)ncell, st) != cudaSuccess)
    return MRI_ECUDA;
  mri_fast_opts o = *opts;
  for (int i = 1; i < 4; ++i) {
    int rc = mri::launch_slow(y, fS + (i - 1) * len, n, grid, st);
    if (rc != MRI_OK) return rc;
    rc = mri_stage_forcing(fS, i, len, k.G[i], phi, stream);
    if (rc != MRI_OK) return rc;
    o.ramp = (i == 1) ? opts->ramp : 0;
    rc = mri_stage_fast_checked(y, p, ncell, phi, 1, (k.c[i] - k.c[i - 1]) * H, h, *m, o, cell_status,
                                cell_stats, n_failed, st, true);
    if (rc != MRI_OK) return rc;
  }
  return MRI_OK;
}

extern "C" const char* mri_status_str(int code) {
  switch (code) {
    case MRI_OK: return "ok";
    case MRI_EINVAL: return "invalid argument";
    case MRI_ENEWTON: return "Newton iteration failed in at least one cell";
    case MRI_ECUDA: return "CUDA error";
    case MRI_ETIMEOUT: return "device work budget exhausted";
    case MRI_ENOMEM: return "workspace too small";
    case MRI_ECONV: return "iterative solve did not converge";
    default: return "unknown status";
  }
}

// ------------------------------------------------------------------ allocation-free step
//
// mri_step_noalloc keeps the step's scratch (three slow evaluations and the stage
// forcing) in one fixed device array that is part of the library image, so a call
// never allocates device memory.  The array is a file-scope __device__ variable:
// every device that loads the library holds it until the process exits.  Host
// code only sees a stand-in for it, so its device address is looked up once per
// device with cudaGetSymbolAddress, with that device current.

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_step_scratch[kStaticScratchBytes];

constexpr int kMaxDevicesCached = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevicesCached] = {};

// Device address of g_step_scratch on the current device (looked up on first use).
int static_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesCached) return MRI_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_step_scratch) != cudaSuccess || p == nullptr) return MRI_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MRI_OK;
}

}  // namespace

extern "C" int mri_step_noalloc(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
                                int mri_method, const mri_mech* mech, const mri_fast_opts* opts,
                                int32_t* cell_status, int32_t* cell_stats, int32_t* n_failed, void* stream) {
  // every argument check of mri_step first, so that an invalid call returns without
  // touching the CUDA runtime (the scratch lookup below runs only for valid calls)
  if (const int rc = mri::step_args_check(y, p, grid, H, h, mri_method, mech, opts)) return rc;
  const mri::Mech* m = reinterpret_cast<const mri::Mech*>(mech);
  const size_t need = mri_step_workspace_size(grid, m->L.n);
  if (need == 0) return MRI_EINVAL;
  if (need > kStaticScratchBytes) return MRI_ENOMEM;   // the grid is too large for the fixed scratch
  void* scratch = nullptr;
  const int rc = static_scratch(&scratch);
  if (rc != MRI_OK) return rc;
  return mri_step(y, p, grid, t, H, h, mri_method, mech, opts, scratch, kStaticScratchBytes, cell_status, cell_stats,
                  n_failed, stream);
}
