// Implicit slow diffusion for IMEX-MRI: the solve-decoupled implicit stage's linear
// system (I - a L) x = b, L = D lap_h the periodic 7-point (2nd-order) Laplacian,
// solved for every component at once by Jacobi-preconditioned conjugate gradients;
// and a first-order IMEX-MRI step built on it (advection explicit in the forcing of
// the fast stage, diffusion implicit in a solve-decoupled correction).
//
// All components share the operator, so the CG recurrences of the n components run
// in lockstep, each with its own scalars.  The Jacobi preconditioner of (I - a L) is
// a constant diagonal, so z = r / diag needs no array.  Every iteration is three
// passes over the state: the stencil apply fused with the per-component partial sums
// of p.Ap, the x / r update fused with the partial sums of r.z, and the direction
// update.  The last block to finish each of the first two passes (a grid-wide arrival
// counter, no waiting) turns the partial sums into alpha and beta, so an iteration is
// three launches.  All sums run in a fixed order (per thread, then over the block's
// cell slots, then over the blocks), so a solve is deterministic.  A component stops updating once its
// residual meets the tolerance; a device "finished" flag turns the launches after
// convergence into no-ops, and the host may read it every few iterations.
#include <cmath>

#include "internal.cuh"

namespace mri {
namespace {

constexpr int kRedBlocks = 1024;    // blocks of the fused passes at most (partial sums per block)
constexpr int kPassThreads = 256;   // threads of a fused pass at least (when that many fit)
constexpr int kPassMax = 1024;      // n <= 1024: one slot of up to 1024 threads
constexpr int kScalThreads = 1024;  // the scalar kernels: one warp per component at a time
constexpr int kDirBlocks = 2432;    // blocks of the direction update (16 per SM)
constexpr int kUnroll = 4;          // cells of a thread's sequence loaded together in the passes

struct Lap7 {
  int nx, ny, nz, n;
  double centre, w[3];   // operator A = I - a L: centre weight and the neighbour weight per axis
  long long st[3];       // element strides of the axes: n, nx n, nx ny n
  long long wrap[3];     // element distance from the first to the last cell of an axis: (N - 1) stride
  unsigned mx, my;       // ceil(2^32 / nx), ceil(2^32 / ny) for the division by nx and ny (0 when 1)
};

// a / d for a < 2^31 with m = ceil(2^32 / d), d >= 2: the product's high word is the
// quotient or one more (a m / 2^32 exceeds a / d by less than 1/2), corrected by the sign
// of the remainder
__device__ __forceinline__ unsigned div_magic(unsigned a, unsigned d, unsigned m) {
  if (m == 0) return a;                       // d == 1
  unsigned q = __umulhi(a, m);
  if ((int)(a - q * d) < 0) --q;
  return q;
}

// Device-side progress of one solve: finished (every component converged) and the
// iterations taken.
struct CgState {
  int finished;
  int iterations;
  unsigned arrive;   // blocks of the current pass that have written their partial sums
};

struct CgScal {          // per component
  double rz, alpha, beta, bb;
  int done;
};

// (A x)[cell][q] for the 7-point operator.  The cell's grid coordinates come from a
// multiply-high division (grids hold at most 2^31 - 1 cells) and the neighbours from the
// element strides of the axes, with a wrap at the periodic boundary.
__device__ __forceinline__ double apply_at(const double* __restrict__ x, const Lap7& s, long long cell, int q) {
  const unsigned cc = (unsigned)cell;
  const unsigned row = div_magic(cc, (unsigned)s.nx, s.mx);
  const unsigned i = cc - row * (unsigned)s.nx;
  const unsigned k = div_magic(row, (unsigned)s.ny, s.my);
  const unsigned j = row - k * (unsigned)s.ny;
  const long long e = cell * s.n + q;
  double acc = s.centre * x[e];
  if (s.nx > 1) {
    const long long ep = e + ((i + 1 == (unsigned)s.nx) ? -s.wrap[0] : s.st[0]);
    const long long em = e + ((i == 0) ? s.wrap[0] : -s.st[0]);
    acc = fma(s.w[0], x[ep] + x[em], acc);
  }
  if (s.ny > 1) {
    const long long ep = e + ((j + 1 == (unsigned)s.ny) ? -s.wrap[1] : s.st[1]);
    const long long em = e + ((j == 0) ? s.wrap[1] : -s.st[1]);
    acc = fma(s.w[1], x[ep] + x[em], acc);
  }
  if (s.nz > 1) {
    const long long ep = e + ((k + 1 == (unsigned)s.nz) ? -s.wrap[2] : s.st[2]);
    const long long em = e + ((k == 0) ? s.wrap[2] : -s.st[2]);
    acc = fma(s.w[2], x[ep] + x[em], acc);
  }
  return acc;
}

// Layout of a fused pass: thread (slot, q) = threadIdx slot rt + q, q < rt = n, slot < S
// (pass_slots); block b takes the cells b S + slot + m (gridDim S).  Consecutive threads
// touch consecutive doubles of the state, and every lane of every full warp has an
// element: the FP64 instructions, which cost the same whatever the active lanes,
// carry no idle lanes.
// The block's partial sums over its slots are written component-major,
// part[q][block], in slot order.
__device__ __forceinline__ void block_partial(double v, int n, int rt, double* __restrict__ part) {
  __shared__ double red[kPassMax];
  const int q = threadIdx.x % rt, slot = threadIdx.x / rt, S = blockDim.x / rt;
  red[threadIdx.x] = v;
  __syncthreads();
  if (slot == 0 && q < n) {
    double s = 0.0;
    for (int k = 0; k < S; ++k) s += red[k * rt + q];
    part[(size_t)q * gridDim.x + blockIdx.x] = s;
  }
}

// sum over the blocks' partials of component q by one warp, in a fixed order (the
// partials of other blocks are read through L2)
__device__ __forceinline__ double sum_parts(const double* part, int nblk, int q, int lane) {
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += __ldcg(part + (size_t)q * nblk + b);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// After a block has written its partial sums: true in the one block that arrives
// last (it then sees every block's partials).  The counter is reset by that block, so
// the next pass starts from zero.  Nothing waits.
__device__ __forceinline__ bool last_block(CgState* cs) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(&cs->arrive, 1u);
    s_last = (t == gridDim.x - 1) ? 1 : 0;
    if (s_last) cs->arrive = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// mode 0: r = b - A x, partial sums of <r, r> and <b, b> (start)
// mode 1: Ap = A p, partial sums of <p, Ap>; the last block sets alpha = <r, z> / <p, A p>
template <int MODE>
__global__ void __launch_bounds__(kPassMax) apply_pass_kernel(const double* __restrict__ x,
                                                                 const double* __restrict__ bvec,
                                                                 double* __restrict__ out, Lap7 s, int rt,
                                                                 double* __restrict__ part1,
                                                                 double* __restrict__ part2, CgScal* sc,
                                                                 CgState* cs) {
  if (MODE == 1 && cs->finished) return;   // uniform over the grid
  const int q = threadIdx.x % rt, slot = threadIdx.x / rt, S = blockDim.x / rt;
  const long long ncell = (long long)s.nx * s.ny * s.nz;
  double a1 = 0.0, a2 = 0.0;
  const long long stride = (long long)gridDim.x * S;
  if (q < s.n)
    for (long long c0 = (long long)blockIdx.x * S + slot; c0 < ncell; c0 += kUnroll * stride) {
      // kUnroll cells of the thread's sequence at once: their loads are in flight
      // together; the sums still run over the cells in sequence order
      double ax[kUnroll], xv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long c = c0 + u * stride;
        ax[u] = (c < ncell) ? apply_at(x, s, c, q) : 0.0;
        xv[u] = (c < ncell) ? (MODE == 0 ? bvec[c * s.n + q] : x[c * s.n + q]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long c = c0 + u * stride;
        if (c >= ncell) break;
        const long long e = c * s.n + q;
        if (MODE == 0) {
          const double rr = xv[u] - ax[u];
          out[e] = rr;
          a1 = fma(rr, rr, a1);
          a2 = fma(xv[u], xv[u], a2);
        } else {
          out[e] = ax[u];
          a1 = fma(xv[u], ax[u], a1);
        }
      }
    }
  block_partial(a1, s.n, rt, part1);
  if (MODE == 0) {
    __syncthreads();
    block_partial(a2, s.n, rt, part2);
    return;
  }
  if (!last_block(cs)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;   // full warps
  for (int qq = warp; warp < nw && qq < s.n; qq += nw) {
    const double pq = sum_parts(part1, gridDim.x, qq, lane);
    if (lane == 0) sc[qq].alpha = (sc[qq].done || !(pq > 0.0)) ? 0.0 : sc[qq].rz / pq;
  }
}

// x += alpha p, r -= alpha Ap, partial sums of <r, r> (components still iterating); the
// last block sets beta = <r, z>_new / <r, z>_old, tests convergence and counts the
// iteration
__global__ void __launch_bounds__(kPassMax) update_pass_kernel(double* __restrict__ x, double* __restrict__ r,
                                                                  const double* __restrict__ p,
                                                                  const double* __restrict__ Ap, long long ncell,
                                                                  int n, int rt, CgScal* sc,
                                                                  double* __restrict__ part, double inv_diag,
                                                                  double tol, CgState* cs) {
  if (cs->finished) return;
  const int q = threadIdx.x % rt, slot = threadIdx.x / rt, S = blockDim.x / rt;
  double acc = 0.0;
  if (q < n && !sc[q].done) {
    const double al = sc[q].alpha;
    const long long stride = (long long)gridDim.x * S;
    for (long long c0 = (long long)blockIdx.x * S + slot; c0 < ncell; c0 += kUnroll * stride) {
      double pv[kUnroll], xv[kUnroll], av[kUnroll], rv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long c = c0 + u * stride;
        const long long e = c * n + q;
        const bool in = c < ncell;
        pv[u] = in ? p[e] : 0.0;
        xv[u] = in ? x[e] : 0.0;
        av[u] = in ? Ap[e] : 0.0;
        rv[u] = in ? r[e] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long c = c0 + u * stride;
        if (c >= ncell) break;
        const long long e = c * n + q;
        x[e] = fma(al, pv[u], xv[u]);
        const double rr = fma(-al, av[u], rv[u]);
        r[e] = rr;
        acc = fma(rr, rr, acc);
      }
    }
  }
  block_partial(acc, n, rt, part);
  if (!last_block(cs)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;   // full warps
  int active = 0;
  for (int qq = warp; warp < nw && qq < n; qq += nw) {
    const double rr = sum_parts(part, gridDim.x, qq, lane);
    CgScal t = sc[qq];
    if (!t.done) {
      const double rz = rr * inv_diag;
      t.beta = (t.rz > 0.0) ? rz / t.rz : 0.0;
      t.rz = rz;
      if (rr <= tol * tol * t.bb) t.done = 1;
    } else {
      t.beta = 0.0;
    }
    __syncwarp();
    if (lane == 0) sc[qq] = t;
    active |= !t.done;
  }
  const int any = __syncthreads_or(active);
  if (threadIdx.x == 0) {
    cs->iterations += 1;
    if (!any) cs->finished = 1;
  }
}

// START: p = r / diag for every component; else p = r / diag + beta p for the
// components still iterating.  Thread (slot, q) of the fused passes' layout owns
// component q of its cells, so the component needs no division.
template <bool START>
__global__ void __launch_bounds__(kPassMax) dir_kernel(double* __restrict__ p, const double* __restrict__ r,
                                                          long long ncell, int n, int rt, double inv_diag,
                                                          const CgScal* sc, const CgState* cs) {
  if (!START && cs->finished) return;
  const int q = threadIdx.x % rt, slot = threadIdx.x / rt, S = blockDim.x / rt;
  if (q >= n) return;
  if (!START && sc[q].done) return;
  const double beta = START ? 0.0 : sc[q].beta;
  const long long stride = (long long)gridDim.x * S;
  for (long long c0 = (long long)blockIdx.x * S + slot; c0 < ncell; c0 += kUnroll * stride) {
    double rv[kUnroll], pv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long c = c0 + u * stride;
      const bool in = c < ncell;
      rv[u] = in ? r[c * n + q] : 0.0;
      pv[u] = (in && !START) ? p[c * n + q] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long c = c0 + u * stride;
      if (c >= ncell) break;
      p[c * n + q] = START ? rv[u] * inv_diag : fma(beta, pv[u], rv[u] * inv_diag);
    }
  }
}

// Start: <r, z> = <r, r> / diag and <b, b>; a component with b = 0 is measured
// against its initial residual.  Convergence: |r|_2 <= tol |b|_2.
__global__ void __launch_bounds__(kScalThreads) cg_init_kernel(const double* part_rr, const double* part_bb, int nblk,
                                                               int n, double inv_diag, double tol, CgScal* sc,
                                                               CgState* cs) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int active = 0;
  for (int q = warp; q < n; q += nw) {
    const double rr = sum_parts(part_rr, nblk, q, lane);
    double bb = sum_parts(part_bb, nblk, q, lane);
    if (!(bb > 0.0)) bb = rr;
    const int done = (rr <= tol * tol * bb) ? 1 : 0;
    if (lane == 0) {
      CgScal s;
      s.rz = rr * inv_diag;
      s.bb = bb;
      s.alpha = 0.0;
      s.beta = 0.0;
      s.done = done;
      sc[q] = s;
    }
    active |= !done;
  }
  const int any = __syncthreads_or(active);
  if (threadIdx.x == 0) {
    cs->finished = any ? 0 : 1;
    cs->iterations = 0;
    cs->arrive = 0u;
  }
}

// info[0] = converged, info[1] = iterations
__global__ void cg_info_kernel(const CgState* cs, int32_t* info) {
  info[0] = cs->finished;
  info[1] = cs->iterations;
}

// cg_info of two solves in a row: converged when both are, iterations summed
__global__ void cg_info_pair_kernel(const int32_t* first, int32_t* info) {
  info[0] = (first[0] != 0 && info[0] != 0) ? 1 : 0;
  info[1] += first[1];
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
  s.st[0] = n;
  s.st[1] = (long long)g->nx * n;
  s.st[2] = (long long)g->nx * g->ny * n;
  s.wrap[0] = (long long)(g->nx - 1) * s.st[0];
  s.wrap[1] = (long long)(g->ny - 1) * s.st[1];
  s.wrap[2] = (long long)(g->nz - 1) * s.st[2];
  s.mx = g->nx > 1 ? (unsigned)(((1ull << 32) + g->nx - 1) / g->nx) : 0u;
  s.my = g->ny > 1 ? (unsigned)(((1ull << 32) + g->ny - 1) / g->ny) : 0u;
  const int N[3] = {g->nx, g->ny, g->nz};
  const double c = g->D / (g->dx * g->dx);
  s.centre = 1.0;
  for (int ax = 0; ax < 3; ++ax) {
    s.w[ax] = (N[ax] > 1) ? -a * c : 0.0;
    if (N[ax] > 1) s.centre += 2.0 * a * c;
  }
  return s;
}

// Slots S of a fused pass (S n threads): at least kPassThreads threads where that many
// fit in kPassMax, and of those the block whose last warp is fullest (fewest idle lanes),
// the smallest on ties.
int pass_slots(int n) {
  const int smax = kPassMax / n;
  int best = smax;
  double best_eff = -1.0;
  for (int S = 1; S <= smax; ++S) {
    const int pt = S * n;
    if (pt < kPassThreads && S < smax) continue;
    const double eff = (double)pt / (double)(((pt + 31) / 32) * 32);
    if (eff > best_eff) { best_eff = eff; best = S; }
  }
  return best;
}

bool grid_ok2(const mri_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->dx > 0 && std::isfinite(g->dx) && g->D >= 0 &&
         std::isfinite(g->D) && (g->order == 2 || g->order == 4) && std::isfinite(g->u[0]) &&
         std::isfinite(g->u[1]) && std::isfinite(g->u[2]) &&
         (long long)g->nx * g->ny * g->nz <= (1ll << 31) - 1;
}

}  // namespace

// The CG solve; ws: 3 len + 2 kRedBlocks n doubles, then n CgScal and the CgState.
// check_every > 0: the host reads the device state every check_every iterations
// (synchronising the stream) and returns once it is finished; check_every = 0: all
// max_iter iterations are enqueued without synchronisation (their launches do nothing
// once the solve is finished), so the sequence can be captured in a CUDA graph.
int diffusion_solve(double* x, const double* b, int n, const mri_grid* g, double a, double tol, int max_iter,
                    int check_every, void* ws, int* iters, int32_t* info, cudaStream_t st) {
  const long long ncell = (long long)g->nx * g->ny * g->nz, len = ncell * n;
  double* r = static_cast<double*>(ws);
  double* p = r + len;
  double* Ap = p + len;
  double* part1 = Ap + len;
  double* part2 = part1 + (size_t)kRedBlocks * n;
  CgScal* sc = reinterpret_cast<CgScal*>(part2 + (size_t)kRedBlocks * n);
  CgState* cs = reinterpret_cast<CgState*>(sc + n);
  const Lap7 op = make_op(g, n, a);
  const double inv_diag = 1.0 / op.centre;
  const int rt = n;
  const int S = pass_slots(n);
  const int pt = S * rt;                                   // threads of a fused pass
  // one wave of the fused passes: as many blocks as stay resident together (at most
  // kRedBlocks, the partial-sum slots), so no block of a pass waits for a second wave
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_pass_kernel<1>, pt, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long long resident = (long long)per_sm * device_sm_count();
  if (resident > kRedBlocks) resident = kRedBlocks;
  const long long want = (ncell + S - 1) / S;
  const int nblk = (int)(want < resident ? want : resident);
  if (iters) *iters = 0;
  apply_pass_kernel<0><<<nblk, pt, 0, st>>>(x, b, r, op, rt, part1, part2, nullptr, nullptr);
  cg_init_kernel<<<1, kScalThreads, 0, st>>>(part1, part2, nblk, n, inv_diag, tol, sc, cs);
  const int dblk = (int)((ncell + S - 1) / S < kDirBlocks ? (ncell + S - 1) / S : kDirBlocks);
  dir_kernel<true><<<dblk, pt, 0, st>>>(p, r, ncell, n, rt, inv_diag, sc, cs);
  if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  CgState h{};
  for (int it = 0; it < max_iter; ++it) {
    if (check_every > 0 && it % check_every == 0) {
      if (cudaMemcpyAsync(&h, cs, sizeof(CgState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return MRI_ECUDA;
      if (h.finished) break;
    }
    apply_pass_kernel<1><<<nblk, pt, 0, st>>>(p, nullptr, Ap, op, rt, part1, nullptr, sc, cs);
    update_pass_kernel<<<nblk, pt, 0, st>>>(x, r, p, Ap, ncell, n, rt, sc, part1, inv_diag, tol, cs);
    dir_kernel<false><<<dblk, pt, 0, st>>>(p, r, ncell, n, rt, inv_diag, sc, cs);
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
  return 3 * len + 2 * (size_t)kRedBlocks * n + (sizeof(CgScal) * (size_t)n + sizeof(CgState) + 7) / 8;
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
  if (const int rc = mri::mech_device_check(*m)) return rc;
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

extern "C" size_t mri_step_imex2_workspace_size(const mri_grid* grid, int n) {
  if (!mri::grid_ok2(grid) || n < 1) return 0;
  const size_t len = (size_t)grid->nx * grid->ny * grid->nz * n;
  // plus the first half step's cg_info (two int32, padded to 16 bytes)
  return 2 * len * sizeof(double) + mri_diffusion_workspace_size(grid, n) + mri_step_workspace_size(grid, n) + 16;
}

namespace mri {
namespace {

// Crank-Nicolson step of the diffusion over 2a: (I - a L) y <- (I + a L) y, from
// x = y; fI and rhs are len-sized scratch
int cn_diffusion(double* y, int n, const mri_grid* gI, double a, double tol, int max_iter, int check_every,
                 double* fI, double* rhs, void* cgws, int* iters, int32_t* info, cudaStream_t st) {
  const long long len = (long long)gI->nx * gI->ny * gI->nz * n;
  int rc = mri_slow_rhs(y, fI, n, gI, 0.0, st);
  if (rc != MRI_OK) return rc;
  axpy_kernel<<<elementwise_blocks(len), 256, 0, st>>>(rhs, y, fI, a, len);
  if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  return diffusion_solve(y, rhs, n, gI, a, tol, max_iter, check_every, cgws, iters, info, st);
}

}  // namespace
}  // namespace mri

extern "C" int mri_step_imex2(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
                              int mri_method, const mri_mech* mech, const mri_fast_opts* opts, double cg_tol,
                              int cg_max_iter, int cg_check_every, void* workspace, size_t workspace_bytes,
                              int32_t* cell_status, int32_t* cell_stats, int32_t* n_failed, int* cg_iterations,
                              int32_t* cg_info, void* stream) {
  if (!mri::grid_ok2(grid) || !mech || !opts || !y || !p || mri_method != MRI_KW3) return MRI_EINVAL;
  if (!(H > 0) || !(h > 0) || !std::isfinite(H) || !std::isfinite(h) || !(cg_tol > 0) || cg_max_iter < 0 ||
      cg_check_every < 0)
    return MRI_EINVAL;
  if (!mri::fast_opts_ok(opts) || opts->time_budget_s != 0.0) return MRI_EINVAL;
  const mri::Mech* m = reinterpret_cast<const mri::Mech*>(mech);
  if (const int rc = mri::mech_device_check(*m)) return rc;
  const int n = m->L.n;
  if (n > 1024) return MRI_EINVAL;
  if (!workspace || workspace_bytes < mri_step_imex2_workspace_size(grid, n)) return MRI_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long len = (long long)grid->nx * grid->ny * grid->nz * n;
  double* fI = static_cast<double*>(workspace);
  double* rhs = fI + len;
  void* cgws = rhs + len;
  void* stepws = static_cast<unsigned char*>(cgws) + mri_diffusion_workspace_size(grid, n);
  int32_t* info1 = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(stepws) + mri_step_workspace_size(grid, n));
  // explicit slow partition of the MRI step: advection (the grid's order); the
  // diffusion is the 7-point Laplacian of the Crank-Nicolson half steps
  mri_grid gE = *grid, gI = *grid;
  gE.D = 0.0;
  gI.u[0] = gI.u[1] = gI.u[2] = 0.0;
  gI.order = 2;
  const double a = 0.25 * H;
  int it1 = 0, it2 = 0;
  // a first half step that misses its tolerance: MRI_ECONV with host checks, and in
  // cg_info (combined with the second half step's) either way
  int rc = mri::cn_diffusion(y, n, &gI, a, cg_tol, cg_max_iter, cg_check_every, fI, rhs, cgws, &it1,
                             cg_info ? info1 : nullptr, st);
  if (rc == MRI_ECONV && cg_info &&
      cudaMemcpyAsync(cg_info, info1, 2 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return MRI_ECUDA;
  if (rc != MRI_OK) return rc;
  rc = mri_step(y, p, &gE, t, H, h, mri_method, mech, opts, stepws, mri_step_workspace_size(grid, n), cell_status,
                cell_stats, n_failed, stream);
  if (rc != MRI_OK) return rc;
  rc = mri::cn_diffusion(y, n, &gI, a, cg_tol, cg_max_iter, cg_check_every, fI, rhs, cgws, &it2, cg_info, st);
  if (cg_iterations) *cg_iterations = (cg_check_every > 0) ? it1 + it2 : -1;
  if (cg_info && (rc == MRI_OK || rc == MRI_ECONV)) {
    mri::cg_info_pair_kernel<<<1, 1, 0, st>>>(info1, cg_info);
    if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  }
  return rc;
}
