// Implicit slow diffusion for IMEX-MRI: the solve-decoupled implicit stage's linear
// system (I - a L) x = b, L = D lap_h the periodic 7-point (2nd-order) Laplacian,
// solved for every component at once by Jacobi-preconditioned conjugate gradients;
// and a first-order IMEX-MRI step built on it (advection explicit in the forcing of
// the fast stage, diffusion implicit in a solve-decoupled correction).
//
// All components share the operator, so the CG recurrences of the n components run
// in lockstep, each with its own scalars: every iteration is a stencil apply, two
// per-component reductions (block partials in fixed order, then a sum over blocks)
// and elementwise updates; a component stops updating once its residual meets the
// tolerance.  The host checks a device "all converged" flag every few iterations.
#include <cmath>

#include "internal.cuh"

namespace mri {
namespace {

constexpr int kRedBlocks = 512;     // blocks of the per-component reductions
constexpr int kCheckEvery = 8;      // iterations between convergence checks on the host

struct Lap7 {
  int nx, ny, nz, n;
  double centre, w[3];   // operator A = I - a L: centre weight and the neighbour weight per axis
};

// Device-side progress of one solve: finished (every component converged), the
// iterations taken and the per-component scalars.  The scalar kernels run as one
// block of one thread per component, so the "any component still iterating" test is
// a block vote and needs no atomics.
struct CgState {
  int finished;
  int iterations;
};

struct CgScal {          // per component
  double rz, alpha, beta, bb;
  int done;
};

// y = A x on [ncell][n]
__global__ void apply_kernel(const double* __restrict__ x, double* __restrict__ y, Lap7 s, const CgState* cs) {
  if (cs && cs->finished) return;
  const long long total = (long long)s.nx * s.ny * s.nz * s.n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cell = e / s.n;
    const int q = (int)(e - cell * s.n);
    const int i = (int)(cell % s.nx), j = (int)((cell / s.nx) % s.ny), k = (int)(cell / ((long long)s.nx * s.ny));
    double acc = s.centre * x[e];
    if (s.nx > 1) {
      const int ip = (i + 1 == s.nx) ? 0 : i + 1, im = (i == 0) ? s.nx - 1 : i - 1;
      acc = fma(s.w[0], x[(((long long)k * s.ny + j) * s.nx + ip) * s.n + q] +
                            x[(((long long)k * s.ny + j) * s.nx + im) * s.n + q], acc);
    }
    if (s.ny > 1) {
      const int jp = (j + 1 == s.ny) ? 0 : j + 1, jm = (j == 0) ? s.ny - 1 : j - 1;
      acc = fma(s.w[1], x[(((long long)k * s.ny + jp) * s.nx + i) * s.n + q] +
                            x[(((long long)k * s.ny + jm) * s.nx + i) * s.n + q], acc);
    }
    if (s.nz > 1) {
      const int kp = (k + 1 == s.nz) ? 0 : k + 1, km = (k == 0) ? s.nz - 1 : k - 1;
      acc = fma(s.w[2], x[(((long long)kp * s.ny + j) * s.nx + i) * s.n + q] +
                            x[(((long long)km * s.ny + j) * s.nx + i) * s.n + q], acc);
    }
    y[e] = acc;
  }
}

// part[block][q] = sum over this block's cells of u[cell][q] * v[cell][q]; thread q of
// the block owns component q (blockDim >= n), so the sums are in a fixed order.
__global__ void dot_partial_kernel(const double* __restrict__ u, const double* __restrict__ v, long long ncell, int n,
                                   double* __restrict__ part, const CgState* cs) {
  if (cs && cs->finished) return;
  const int q = threadIdx.x;
  if (q >= n) return;
  double acc = 0.0;
  for (long long c = blockIdx.x; c < ncell; c += gridDim.x) acc = fma(u[c * n + q], v[c * n + q], acc);
  part[(size_t)blockIdx.x * n + q] = acc;
}

__device__ __forceinline__ double sum_parts(const double* part, int nblk, int n, int q) {
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * n + q];
  return s;
}

// after r = b - A x and z = r / diag: rz = <r, z>, bb = <b, b> (both from partials).
// One block, thread q = component q.
__global__ void cg_init_kernel(const double* part_rz, const double* part_bb, int nblk, int n, double diag, double tol,
                               CgScal* sc, CgState* cs) {
  const int q = threadIdx.x;
  bool active = false;
  if (q < n) {
    CgScal s;
    s.rz = sum_parts(part_rz, nblk, n, q);
    s.bb = sum_parts(part_bb, nblk, n, q);
    s.alpha = s.beta = 0.0;
    // Jacobi: z = r / diag, so |r|^2 = diag <r, z>.  The residual is measured against
    // |b|; a component with b = 0 is measured against its initial residual instead.
    if (!(s.bb > 0.0)) s.bb = s.rz * diag;
    s.done = (s.rz * diag <= tol * tol * s.bb) ? 1 : 0;
    sc[q] = s;
    active = !s.done;
  }
  const int any = __syncthreads_or(active);
  if (q == 0) {
    cs->finished = any ? 0 : 1;
    cs->iterations = 0;
  }
}

// alpha = <r, z> / <p, A p>
__global__ void cg_alpha_kernel(const double* part_pq, int nblk, int n, CgScal* sc, const CgState* cs) {
  if (cs->finished) return;
  const int q = threadIdx.x;
  if (q >= n) return;
  const double pq = sum_parts(part_pq, nblk, n, q);
  sc[q].alpha = (sc[q].done || !(pq > 0.0)) ? 0.0 : sc[q].rz / pq;
}

// x += alpha p; r -= alpha A p; z = r / diag
__global__ void cg_update_kernel(double* x, double* r, double* z, const double* p, const double* Ap, long long len,
                                 int n, double inv_diag, const CgScal* sc, const CgState* cs) {
  if (cs->finished) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % n);
    const double al = sc[q].alpha;
    x[e] = fma(al, p[e], x[e]);
    const double rr = fma(-al, Ap[e], r[e]);
    r[e] = rr;
    z[e] = rr * inv_diag;
  }
}

// beta = <r, z>_new / <r, z>_old; convergence on |r|^2 = diag <r, z>.  One block.
__global__ void cg_beta_kernel(const double* part_rz, int nblk, int n, double diag, double tol, CgScal* sc,
                               CgState* cs) {
  if (cs->finished) return;     // uniform over the block: read before anyone writes
  const int q = threadIdx.x;
  bool active = false;
  if (q < n) {
    CgScal s = sc[q];
    if (!s.done) {
      const double rz = sum_parts(part_rz, nblk, n, q);
      s.beta = (s.rz > 0.0) ? rz / s.rz : 0.0;
      s.rz = rz;
      if (rz * diag <= tol * tol * s.bb) s.done = 1;
    } else {
      s.beta = 0.0;
    }
    sc[q] = s;
    active = !s.done;
  }
  const int any = __syncthreads_or(active);
  if (q == 0) {
    cs->iterations += 1;
    if (!any) cs->finished = 1;
  }
}

// p = z + beta p (components still iterating)
__global__ void cg_dir_kernel(double* p, const double* z, long long len, int n, const CgScal* sc, const CgState* cs) {
  if (cs->finished) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % n);
    if (!sc[q].done) p[e] = fma(sc[q].beta, p[e], z[e]);
  }
}

// r = b - r (r holds A x on entry), z = r / diag, p = z
__global__ void cg_start_kernel(const double* b, double* r, double* z, double* p, long long len, double inv_diag) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const double rr = b[e] - r[e];
    r[e] = rr;
    const double zz = rr * inv_diag;
    z[e] = zz;
    p[e] = zz;
  }
}

// info[0] = converged, info[1] = iterations
__global__ void cg_info_kernel(const CgState* cs, int32_t* info) {
  info[0] = cs->finished;
  info[1] = cs->iterations;
}

// out = u + s v
__global__ void axpy_kernel(double* out, const double* u, const double* v, double s, long long len) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = fma(s, v[e], u[e]);
}

int elementwise_blocks(long long len) {
  long long b = (len + 255) / 256;
  const long long cap = (long long)device_sm_count() * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

Lap7 make_op(const mri_grid* g, int n, double a) {
  Lap7 s{};
  s.nx = g->nx; s.ny = g->ny; s.nz = g->nz; s.n = n;
  const int N[3] = {g->nx, g->ny, g->nz};
  const double c = g->D / (g->dx * g->dx);
  s.centre = 1.0;
  for (int ax = 0; ax < 3; ++ax) {
    s.w[ax] = (N[ax] > 1) ? -a * c : 0.0;
    if (N[ax] > 1) s.centre += 2.0 * a * c;
  }
  return s;
}

bool grid_ok2(const mri_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->dx > 0 && std::isfinite(g->dx) && g->D >= 0 &&
         std::isfinite(g->D) && (g->order == 2 || g->order == 4) && std::isfinite(g->u[0]) &&
         std::isfinite(g->u[1]) && std::isfinite(g->u[2]) &&
         (long long)g->nx * g->ny * g->nz <= (1ll << 31) - 1;
}

}  // namespace

// The CG solve; ws: 4 len + kRedBlocks (2 n) doubles, then n CgScal and the CgState.
// check_every > 0: the host reads the device state every check_every iterations
// (synchronising the stream) and returns once it is finished; check_every = 0: all
// max_iter iterations are enqueued without synchronisation (their launches do nothing
// once the solve is finished), so the sequence can be captured in a CUDA graph.
int diffusion_solve(double* x, const double* b, int n, const mri_grid* g, double a, double tol, int max_iter,
                    int check_every, void* ws, int* iters, int32_t* info, cudaStream_t st) {
  const long long ncell = (long long)g->nx * g->ny * g->nz, len = ncell * n;
  double* r = static_cast<double*>(ws);
  double* z = r + len;
  double* p = z + len;
  double* Ap = p + len;
  double* part1 = Ap + len;
  double* part2 = part1 + (size_t)kRedBlocks * n;
  CgScal* sc = reinterpret_cast<CgScal*>(part2 + (size_t)kRedBlocks * n);
  CgState* cs = reinterpret_cast<CgState*>(sc + n);
  const Lap7 op = make_op(g, n, a);
  const double diag = op.centre, inv_diag = 1.0 / op.centre;
  const int eb = elementwise_blocks(len);
  const int nblk = (int)(ncell < kRedBlocks ? ncell : kRedBlocks);
  const int rt = ((n + 31) / 32) * 32;
  if (iters) *iters = 0;
  apply_kernel<<<eb, 256, 0, st>>>(x, r, op, nullptr);
  cg_start_kernel<<<eb, 256, 0, st>>>(b, r, z, p, len, inv_diag);
  // the initial reductions run unconditionally: cs is first written by cg_init
  dot_partial_kernel<<<nblk, rt, 0, st>>>(r, z, ncell, n, part1, nullptr);
  dot_partial_kernel<<<nblk, rt, 0, st>>>(b, b, ncell, n, part2, nullptr);
  cg_init_kernel<<<1, rt, 0, st>>>(part1, part2, nblk, n, diag, tol, sc, cs);
  if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  CgState h{};
  for (int it = 0; it < max_iter; ++it) {
    if (check_every > 0 && it % check_every == 0) {
      if (cudaMemcpyAsync(&h, cs, sizeof(CgState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return MRI_ECUDA;
      if (h.finished) break;
    }
    apply_kernel<<<eb, 256, 0, st>>>(p, Ap, op, cs);
    dot_partial_kernel<<<nblk, rt, 0, st>>>(p, Ap, ncell, n, part1, cs);
    cg_alpha_kernel<<<1, rt, 0, st>>>(part1, nblk, n, sc, cs);
    cg_update_kernel<<<eb, 256, 0, st>>>(x, r, z, p, Ap, len, n, inv_diag, sc, cs);
    dot_partial_kernel<<<nblk, rt, 0, st>>>(r, z, ncell, n, part1, cs);
    cg_beta_kernel<<<1, rt, 0, st>>>(part1, nblk, n, diag, tol, sc, cs);
    cg_dir_kernel<<<eb, 256, 0, st>>>(p, z, len, n, sc, cs);
    if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  }
  if (info) {
    cg_info_kernel<<<1, 1, 0, st>>>(cs, info);
    if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  }
  if (check_every == 0) return MRI_OK;
  if (cudaMemcpyAsync(&h, cs, sizeof(CgState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MRI_ECUDA;
  if (iters) *iters = h.iterations;
  return h.finished ? MRI_OK : MRI_ECONV;
}

size_t diffusion_ws_doubles(const mri_grid* g, int n) {
  const size_t len = (size_t)g->nx * g->ny * g->nz * n;
  return 4 * len + 2 * (size_t)kRedBlocks * n + (sizeof(CgScal) * (size_t)n + sizeof(CgState) + 7) / 8;
}

}  // namespace mri

extern "C" size_t mri_diffusion_workspace_size(const mri_grid* grid, int n) {
  if (!mri::grid_ok2(grid) || n < 1) return 0;
  return mri::diffusion_ws_doubles(grid, n) * sizeof(double);
}

extern "C" int mri_diffusion_solve(double* x, const double* b, int n, const mri_grid* grid, double a, double tol,
                                   int max_iter, int check_every, void* workspace, size_t workspace_bytes,
                                   int* iterations, int32_t* cg_info, void* stream) {
  if (!mri::grid_ok2(grid) || n < 1 || n > 1024 || !x || !b || !(a >= 0) || !std::isfinite(a) || !(tol > 0) ||
      max_iter < 0 || check_every < 0)
    return MRI_EINVAL;
  if (!workspace || workspace_bytes < mri_diffusion_workspace_size(grid, n)) return MRI_ENOMEM;
  return mri::diffusion_solve(x, b, n, grid, a, tol, max_iter, check_every, workspace, iterations, cg_info,
                              static_cast<cudaStream_t>(stream));
}

extern "C" size_t mri_step_imex1_workspace_size(const mri_grid* grid, int n) {
  if (!mri::grid_ok2(grid) || n < 1) return 0;
  const size_t len = (size_t)grid->nx * grid->ny * grid->nz * n;
  return (2 * len) * sizeof(double) + mri_diffusion_workspace_size(grid, n);
}

extern "C" int mri_step_imex1(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
                              const mri_mech* mech, const mri_fast_opts* opts, double cg_tol, int cg_max_iter,
                              int cg_check_every, void* workspace, size_t workspace_bytes, int32_t* cell_status,
                              int32_t* cell_stats, int32_t* n_failed, int* cg_iterations, int32_t* cg_info,
                              void* stream) {
  if (!mri::grid_ok2(grid) || !mech || !opts || !y || !p) return MRI_EINVAL;
  if (!(H > 0) || !(h > 0) || !std::isfinite(H) || !std::isfinite(h) || !(cg_tol > 0) || cg_max_iter < 0 ||
      cg_check_every < 0)
    return MRI_EINVAL;
  if (!mri::fast_opts_ok(opts) || opts->time_budget_s != 0.0) return MRI_EINVAL;
  const mri::Mech* m = reinterpret_cast<const mri::Mech*>(mech);
  const int n = m->L.n;
  if (n > 1024) return MRI_EINVAL;
  if (!workspace || workspace_bytes < mri_step_imex1_workspace_size(grid, n)) return MRI_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long ncell = (long long)grid->nx * grid->ny * grid->nz, len = ncell * n;
  double* fI = static_cast<double*>(workspace);
  double* phi = fI + len;
  void* cgws = phi + len;
  // explicit partition: advection (the grid's order); implicit: diffusion on the 7-point
  // Laplacian, the operator the implicit solve inverts
  mri_grid gE = *grid, gI = *grid;
  gE.D = 0.0;
  gI.u[0] = gI.u[1] = gI.u[2] = 0.0;
  gI.order = 2;
  int rc = mri_slow_rhs(y, phi, n, &gE, t, stream);
  if (rc != MRI_OK) return rc;
  if ((rc = mri_slow_rhs(y, fI, n, &gI, t, stream)) != MRI_OK) return rc;
  const int eb = mri::elementwise_blocks(len);
  mri::axpy_kernel<<<eb, 256, 0, st>>>(phi, phi, fI, 1.0, len);   // forcing f^E(y_n) + f^I(y_n)
  if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  if (cell_status && cudaMemsetAsync(cell_status, 0, sizeof(int32_t) * (size_t)ncell, st) != cudaSuccess)
    return MRI_ECUDA;
  rc = mri::mri_stage_fast_checked(y, p, (int)ncell, phi, 1, H, h, *m, *opts, cell_status, cell_stats, n_failed, st,
                                   true);
  if (rc != MRI_OK) return rc;
  // solve-decoupled implicit correction: (I - H L) y_{n+1} = v - H L y_n, from x = v
  mri::axpy_kernel<<<eb, 256, 0, st>>>(phi, y, fI, -H, len);
  if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  return mri::diffusion_solve(y, phi, n, &gI, H, cg_tol, cg_max_iter, cg_check_every, cgws, cg_iterations, cg_info,
                              st);
}
