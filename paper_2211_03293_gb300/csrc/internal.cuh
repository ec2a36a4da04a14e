// Internal declarations shared by the translation units of libmri (the CUDA
// product path).  Nothing here is visible through the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mri.h"

namespace mri {

constexpr double kRu = 8.314462618;          // J/(mol K)
constexpr double kPatm = 101325.0;           // Pa, standard-state pressure of K_c
constexpr double kLn10 = 2.30258509299404568401799145468;
constexpr int kMaxSpecies = 127;
constexpr int kMaxReactions = 1023;
constexpr int kMaxK = 4;                     // forcing polynomial terms
constexpr int kMaxWarps = 12;                // warps (cells in flight) per CTA
constexpr int kTroeSlots = 12;               // per-cell doubles of one falloff reaction's intermediates

// Byte offsets of the sections of the mechanism table.  The table is one
// contiguous device buffer that every CTA copies into shared memory.  Species
// vectors have a pad slot at index Ns (concentration 1, Gibbs/enthalpy 0) that
// absent reaction partners point to, so rate products need no branches.
struct Layout {
  int Ns, R, n, n_eff, n_troe, n_tb;  // n = Ns + 1; n_tb = reactions with [M]
  int nsv;          // species-vector length incl. pad slot, even
  int rv;           // reaction-vector length, even
  // table sections (bytes from the start of the table)
  int o_cp, o_h, o_s;     // double [5][nsv] cp/R, h/RT, s/R polynomial coefficients (SoA)
  int o_h5, o_s6;         // double [nsv] a6 (enthalpy const), a7 (entropy const)
  int o_dcp;              // double [4][nsv] coefficients of d(cp/R)/dT
  int o_W, o_invW;        // double [nsv]
  int o_lnA, o_b, o_Ta;   // double [rv]
  int o_rxn;              // uint64 [rv]: bytes 0-2 reactants, 3-5 products (pad = Ns), 6 dn (int8), 7 type
  int o_rrow;             // int32 [rv]: eff row (low 16 bits, 0xffff none) | troe row << 16
  int o_eptr;             // int32 [n_eff + 1] sparse (alpha - 1) lists
  int o_eidx;             // int32 [ne]
  int o_eval;             // double [ne]
  int o_troe;             // double [n_troe][8]: lnA0, b0, Ta0, a, 1/T***, 1/T*, T**, 0
  int o_gent;             // int32 [n_went]: r (10 bits) | nu + 8 (4) | slot (8) | run-end flag (1)
  int o_gsptr;            // int32 [Ns + 1] species -> partial-sum slots
  int o_gslot;            // int32 [..] slot indices
  int g_chunk, n_went, n_slots;   // entries per lane, list length, partial-sum slots
  int o_cptr;             // int32 [Ns + 1] Jacobian column -> reaction entries
  int o_cent;             // uint64 [nc]: r (16) | mult_f (4) | mult_r (4) | o1..o4 (8 bits each)
  int o_rsp;              // uint64 [rv][2]: word 0 species k0..k5 + count; word 1 int8 nu0..nu5
  int o_tbl;              // int32 [n_tb]: reactions with an efficiency row (third body or falloff)
  int o_tcptr;            // int32 [Ns + 1] Jacobian column -> third-body corrections
  int o_tcr;              // int32 [ntc]: reaction of the correction
  int o_tcv, o_tcv32;     // double / float [ntc]: alpha_rl - 1
  int o_trx;              // int32 [n_troe]: reaction index of each falloff row
  int o_exp2;             // double [kExpTab]: 2^(j/128), the table of the exponential (fastmath.cuh)
  int o_logt;             // double [260]: 1/F, log F, ln2 split: the table of the logarithm (fastmath.cuh)
  int o_nu;               // double [8]: the small integers -3..4 as doubles (index v + 3), so kernels
                          // turn stoichiometric integers into doubles with a load, not a conversion
  // FP32 copies of the constants the mixed-precision Jacobian reads
  int o_nu32;             // float [8]
  int o_W32, o_invW32;    // float [nsv]
  int o_dcp32;            // float [4][nsv]
  int bytes;              // total, multiple of 16
  // per-cell workspace (doubles) inside shared memory
  int ld;                 // leading dimension of the n x n matrix (odd)
  int ws_doubles;         // doubles per cell (warp), FP64 form, K = kMaxK
  int ws_doubles32;       // doubles per cell (warp), mixed-precision form, K = kMaxK
};

// Newton-matrix cache entry: header, then the factorised matrix (n * ld values: LU
// factors, or with layout 1 the transposed inverse), the diagonal inverses (n values;
// unused by layout 1) and the pivot permutation (n int32), in the form's precision,
// then (8-byte aligned) f^F at the cell's state when the last call ended (n doubles;
// has_f = 1 when present).
struct McHeader {
  double hg;
  int age, tag, n, prec;
  int has_f;
  int layout;   // 0: LU factors, 1: transposed inverse (MRI_LU_INVERSE)
};
constexpr int kMcTag = 0x4D434145;   // marks a filled entry (a zeroed entry is empty)

__host__ __device__ inline size_t mc_f_offset(const Layout& L, bool prec32) {
  const size_t vb = prec32 ? 4 : 8;
  const size_t b = sizeof(McHeader) + (size_t)L.n * L.ld * vb + (size_t)L.n * vb + (size_t)L.n * 4;
  return (b + 7) / 8 * 8;
}

__host__ __device__ inline size_t mc_stride(const Layout& L, bool prec32) {
  const size_t b = mc_f_offset(L, prec32) + (size_t)L.n * 8;
  return (b + 127) / 128 * 128;
}

// Work-queue counters per mechanism: one per stage launch in flight.  Eager launches
// take theirs from one ring and launches recorded under stream capture from a second
// one, so a CUDA graph, which keeps its counter for as long as it lives, never shares
// a counter with an eager launch.
constexpr int kQueueSlots = 256;        // eager launches
constexpr int kGraphQueueSlots = 256;   // launches recorded into graphs

struct Mech {             // what mri_mech points at
  Layout L;
  void* d_table = nullptr;   // device copy of the table
  int* d_queue = nullptr;    // kQueueSlots + kGraphQueueSlots work-queue counters
  unsigned queue_next = 0;   // next eager counter to hand out (round robin)
  unsigned graph_next = 0;   // next captured-launch counter to hand out (round robin)
  int device = -1;
};

// Per-cell workspace carve-up (double offsets inside the warp's region).  With
// prec32 (the mixed-precision form) the Newton matrix and its factors are FP32 and a
// float region holds FP32 copies of the Jacobian inputs.
struct WsOffsets {
  int M, y0, Z, d, res, F0, F1, Fl, r, f, base, phi, C, hh, cp, wd, DT, DC, aux, dinv, piv;
  int q, kfw, krw, dqdT, tbs;
  int E, Einv, c0p, tro, tbk;
  int f32;     // start of the float region (prec32 only), in doubles
  int r32;     // prec32: 1 when the FP32 k_f, k_r and third-body scales live in q and tro
  int total;
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// float offsets inside the f32 region
struct F32Offsets {
  int C, hh, cp, wd, DT, DC, aux, tbk, kfw, krw, tbs, d, dinv, total;
};

// compact: without the per-reaction FP32 arrays (kfw, krw, tbs), the Jacobian's
// column vectors (DC, aux) and the FP32 correction (d), which then live in dead FP64
// scratch (WsOffsets::r32).
__host__ __device__ inline F32Offsets f32_offsets(const Layout& L, bool compact = false) {
  F32Offsets f;
  const int nv = round_up(L.n + 1, 4), ns = round_up(L.nsv, 4), rv = round_up(L.rv, 4);
  int o = 0;
  f.C = o; o += ns;
  f.hh = o; o += ns;
  f.cp = o; o += ns;
  f.wd = o; o += ns;
  f.DT = o; o += ns;
  f.tbk = o; o += ns;
  f.DC = f.aux = f.kfw = f.krw = f.tbs = f.d = -1;
  if (!compact) {
    f.DC = o; o += ns;
    f.aux = o; o += ns;
    f.kfw = o; o += rv;
    f.krw = o; o += rv;
    f.tbs = o; o += rv;
    f.d = o; o += nv;
  }
  f.dinv = o; o += nv;
  f.total = round_up(o, 4);
  return f;
}

// matrix = false: no Newton matrix (the explicit fast methods need none); every other
// section keeps its meaning.
__host__ __device__ inline WsOffsets ws_offsets(const Layout& L, bool prec32 = false, int K = kMaxK,
                                                bool matrix = true) {
  WsOffsets w;
  int nv = round_up(L.n + 1, 2);
  int o = 0;
  w.M = o;
  if (matrix) o += prec32 ? round_up(L.n * L.ld, 4) / 2 : round_up(L.n * L.ld, 2);
  w.y0 = o; o += nv;
  w.Z = o; o += nv;
  w.d = o; o += nv;
  w.res = o; o += nv;
  w.F0 = o; o += nv;
  w.F1 = o; o += nv;
  w.Fl = o; o += nv;
  w.r = o; o += nv;
  w.f = -1;   // f^F of the explicit methods and the per-kernel entries (the stage solve forms it in place)
  if (!prec32) { w.f = o; o += nv; }
  w.base = o; o += nv;
  w.C = o; o += L.nsv;
  w.hh = o; o += L.nsv;
  w.cp = o; o += L.nsv;
  w.wd = o; o += L.nsv;
  w.DT = o; o += L.nsv;
  w.dinv = o; o += prec32 ? 0 : nv;   // FP64 pivots' inverses (the FP32 form keeps its own)
  w.piv = o; o += nv / 2 + 1;   // int32 pivots
  o = round_up(o, 2);
  w.q = o; o += L.rv;
  if (prec32 && 4 * L.rv <= w.y0 - w.M) {
    // mixed form: the FP64 per-reaction Jacobian inputs are dead once their FP32
    // copies exist, before the FP32 Newton matrix is assembled, so they share its
    // storage (the previous factorisation is being replaced at that point)
    w.kfw = w.M; w.krw = w.M + L.rv; w.dqdT = w.M + 2 * L.rv; w.tbs = w.M + 3 * L.rv;
  } else {
    w.kfw = o; o += L.rv;
    w.krw = o; o += L.rv;
    w.dqdT = o; o += L.rv;
    w.tbs = o; o += L.rv;
  }
  w.E = o; o += L.nsv;
  w.Einv = o; o += L.nsv;
  // the Jacobian's DC and column-sum vectors reuse E and 1/E, which only the rate
  // pass before it reads
  w.DC = w.E;
  w.aux = w.Einv;
  w.c0p = o; o += 6;
  // falloff intermediates; after the reaction pass the same doubles hold the
  // partial sums of the balanced production-rate pass
  w.tro = o;
  {
    const int ntro = kTroeSlots * (L.n_troe > 0 ? L.n_troe : 1);
    o += ntro > L.n_slots ? ntro : L.n_slots;
  }
  w.tbk = o; o += L.nsv;
  o = round_up(o, 2);
  // mixed form: the FP32 copies of k_f, k_r and the third-body scales are made after
  // the Jacobian's rate pass has summed its production rates, when the rates (q, rv
  // doubles: room for both rv-float copies) and the falloff / partial-sum scratch
  // (tro) are dead, so they live there when tro holds rv floats; the FP32 Jacobian's
  // DC and column-sum vectors take E and 1/E as the FP64 ones do, and the FP32 Newton
  // correction, made while no rates are live, takes q too
  {
    const int ntro = kTroeSlots * (L.n_troe > 0 ? L.n_troe : 1);
    const int tro_doubles = ntro > L.n_slots ? ntro : L.n_slots;
    w.r32 = (prec32 && 2 * tro_doubles >= L.rv && 2 * L.rv >= round_up(L.n + 1, 4)) ? 1 : 0;
  }
  w.f32 = o;
  if (prec32) o += f32_offsets(L, w.r32 != 0).total / 2;
  w.phi = o; o += K * nv;        // forcing coefficients: sized by the launch's K
  w.total = round_up(o, 2);
  return w;
}

// launch helpers implemented in fast.cu / slow.cu
int launch_stage_fast(double* y, const double* p, int ncell, const double* phi, int K, double Hs, double h,
                      const Mech& m, const mri_fast_opts& o, int ramp, int32_t* status, int32_t* stats,
                      int32_t* n_failed, cudaStream_t st, bool sticky, const double* guess = nullptr,
                      int start = MRI_START_PREDICTOR, int32_t* n_fallback = nullptr,
                      const int8_t* step_exp = nullptr);
bool fast_opts_ok(const mri_fast_opts* o);
bool is_explicit(int method);
// MRI_OK when the current device is the one the mechanism's tables were loaded on,
// MRI_EINVAL when it is another, MRI_ECUDA when the device cannot be queried
int mech_device_check(const Mech& m);
// mri_stage_fast after the pointer checks; sticky = write only failing statuses
int mri_stage_fast_checked(double* y, const double* p, int ncell, const double* phi, int K, double Hstage,
                           double h, const Mech& m, const mri_fast_opts& o, int32_t* cell_status,
                           int32_t* cell_stats, int32_t* n_failed, cudaStream_t st, bool sticky);
int device_smem_limit();
int device_sm_count();
int diffusion_solve(double* x, const double* b, int n, const mri_grid* g, double a, double tol, int max_iter,
                    int check_every, void* ws, int* iters, int32_t* info, cudaStream_t st);

}  // namespace mri
