// The fast-partition hot path: chemistry right-hand side, analytic Jacobian,
// warp-cooperative dense LU and the SDIRK / Newton substep driver.
//
// Organisation: one warp owns one grid cell for a whole MRI stage.  The
// mechanism table lives in shared memory (one copy per CTA); each warp has a
// private shared-memory workspace with the cell's n x n Newton matrix and the
// vectors of the stage.  Lanes split reactions (rates), species (sums over
// reactions), Jacobian columns (assembly) and matrix rows/entries (LU).  All
// arithmetic of the state, residual, rates and factorisation is FP64.
#include <cmath>
#include <cstdio>

#include "internal.cuh"

namespace mri {

// ------------------------------------------------------------------ views

struct Tab {
  const double *cp, *hh, *ss, *h5, *s6, *dcp, *W, *invW, *lnA, *b, *Ta, *effd, *eval, *troe, *nu;
  const uint64_t *rxn, *cent, *rsp;
  const int32_t *rrow, *eptr, *eidx, *wptr, *went, *cptr, *tbl;
  int Ns, R, n, nsv, n_tb;
  __device__ Tab(const unsigned char* s, const Layout& L) {
    cp = reinterpret_cast<const double*>(s + L.o_cp);
    hh = reinterpret_cast<const double*>(s + L.o_h);
    ss = reinterpret_cast<const double*>(s + L.o_s);
    h5 = reinterpret_cast<const double*>(s + L.o_h5);
    s6 = reinterpret_cast<const double*>(s + L.o_s6);
    dcp = reinterpret_cast<const double*>(s + L.o_dcp);
    W = reinterpret_cast<const double*>(s + L.o_W);
    invW = reinterpret_cast<const double*>(s + L.o_invW);
    lnA = reinterpret_cast<const double*>(s + L.o_lnA);
    b = reinterpret_cast<const double*>(s + L.o_b);
    Ta = reinterpret_cast<const double*>(s + L.o_Ta);
    effd = reinterpret_cast<const double*>(s + L.o_effd);
    eval = reinterpret_cast<const double*>(s + L.o_eval);
    troe = reinterpret_cast<const double*>(s + L.o_troe);
    nu = reinterpret_cast<const double*>(s + L.o_nu) + 3;   // nu[v] for v in -3..4
    rxn = reinterpret_cast<const uint64_t*>(s + L.o_rxn);
    cent = reinterpret_cast<const uint64_t*>(s + L.o_cent);
    rsp = reinterpret_cast<const uint64_t*>(s + L.o_rsp);
    rrow = reinterpret_cast<const int32_t*>(s + L.o_rrow);
    eptr = reinterpret_cast<const int32_t*>(s + L.o_eptr);
    eidx = reinterpret_cast<const int32_t*>(s + L.o_eidx);
    wptr = reinterpret_cast<const int32_t*>(s + L.o_wptr);
    went = reinterpret_cast<const int32_t*>(s + L.o_went);
    cptr = reinterpret_cast<const int32_t*>(s + L.o_cptr);
    tbl = reinterpret_cast<const int32_t*>(s + L.o_tbl);
    Ns = L.Ns; R = L.R; n = L.n; nsv = L.nsv; n_tb = L.n_tb;
  }
};

struct WS {
  double *M, *y0, *Z, *d, *res, *F[2], *r, *f, *base, *phi, *C, *g, *hh, *cp, *wd, *DT, *DC, *aux, *dinv;
  int* piv;
  double *q, *kfw, *krw, *dqdT, *tbs;
  int ld, nv;
  __device__ WS(double* base, const Layout& L) {
    WsOffsets o = ws_offsets(L);
    M = base + o.M; y0 = base + o.y0; Z = base + o.Z; d = base + o.d;
    F[0] = base + o.F0; F[1] = base + o.F1; r = base + o.r; f = base + o.f; phi = base + o.phi;
    this->base = base + o.base;
    res = base + o.res;
    C = base + o.C; g = base + o.g; hh = base + o.hh; cp = base + o.cp; wd = base + o.wd;
    DT = base + o.DT; DC = base + o.DC; aux = base + o.aux; dinv = base + o.dinv;
    piv = reinterpret_cast<int*>(base + o.piv);
    q = base + o.q; kfw = base + o.kfw; krw = base + o.krw; dqdT = base + o.dqdT; tbs = base + o.tbs;
    ld = L.ld;
    nv = round_up(L.n + 1, 2);
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// Copy the mechanism table (global) into shared memory with 16-byte loads.
__device__ void stage_table(unsigned char* dst, const unsigned char* src, int bytes) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

// ------------------------------------------------------------------ chemistry

struct Scal {        // warp-uniform per-evaluation scalars
  double T, invT, lnT, S, rho, invrho, Ctot, cpm, Q;
};

// Species concentrations, NASA-7 thermo, rates of progress, production rates and
// f^F at state Z (Y_1..Y_Ns, T).  With JAC also the per-reaction pieces of the
// Jacobian: [M]-weighted k_f, k_r, d q / d T, the third-body scale and
// sum_r nu dq/dT per species.
template <bool JAC>
__device__ __forceinline__ void chem_eval(const Tab& t, const WS& w, const double* Z, double p, Scal& s, int lane) {
  const int Ns = t.Ns, R = t.R, nsv = t.nsv;
  const double T = Z[Ns];
  double part = 0.0;
  for (int k = lane; k < Ns; k += 32) part = fma(Z[k], t.invW[k], part);
  const double S = warp_sum(part);
  const double invT = 1.0 / T;
  const double lnT = log(T);
  const double rho = p / (kRu * T * S);
  const double invrho = kRu * T * S / p;
  double ctot = 0.0;
  for (int k = lane; k < Ns; k += 32) {
    double c = rho * Z[k] * t.invW[k];
    w.C[k] = c;
    ctot += c;
    double cpv = fma(fma(fma(fma(t.cp[4 * nsv + k], T, t.cp[3 * nsv + k]), T, t.cp[2 * nsv + k]), T,
                         t.cp[nsv + k]), T, t.cp[k]);
    double hv = fma(fma(fma(fma(t.hh[4 * nsv + k], T, t.hh[3 * nsv + k]), T, t.hh[2 * nsv + k]), T,
                        t.hh[nsv + k]), T, t.hh[k]) + t.h5[k] * invT;
    double sv = fma(fma(fma(fma(t.ss[4 * nsv + k], T, t.ss[3 * nsv + k]), T, t.ss[2 * nsv + k]), T,
                        t.ss[nsv + k]), T, fma(t.ss[k], lnT, t.s6[k]));
    w.cp[k] = cpv;
    w.hh[k] = hv;
    w.g[k] = hv - sv;
  }
  if (lane == 0) { w.C[Ns] = 1.0; w.g[Ns] = 0.0; w.hh[Ns] = 0.0; }
  const double Ctot = warp_sum(ctot);
  __syncwarp();
  const double lnC0 = 9.4080919689617464985 - lnT;   // ln(p_atm / R_u) - ln T
  for (int r = lane; r < R; r += 32) {
    const uint64_t rec = t.rxn[r];
    const int i0 = rec & 0xff, i1 = (rec >> 8) & 0xff, i2 = (rec >> 16) & 0xff;
    const int j0 = (rec >> 24) & 0xff, j1 = (rec >> 32) & 0xff, j2 = (rec >> 40) & 0xff;
    const int dn = (int)(int8_t)((rec >> 48) & 0xff);
    const int type = (int)(rec >> 56);
    const double sumg = (w.g[j0] + w.g[j1] + w.g[j2]) - (w.g[i0] + w.g[i1] + w.g[i2]);
    const double lnKc = fma(t.nu[dn], lnC0, -sumg);
    const double lnkinf = fma(t.b[r], lnT, t.lnA[r]) - t.Ta[r] * invT;
    double kf = exp(lnkinf);
    double M = 0.0, dlnkf_dT = 0.0, dlnkf_dM = 0.0;
    if (JAC) dlnkf_dT = fma(t.Ta[r], invT, t.b[r]) * invT;
    if (type != 0) {
      const int row = t.rrow[r] & 0xffff;
      M = Ctot;
      for (int e = t.eptr[row]; e < t.eptr[row + 1]; ++e) M = fma(t.eval[e], w.C[t.eidx[e]], M);
    }
    if (type == 2) {
      // Lindemann falloff with Troe broadening: Pr = k0 [M] / k_inf,
      // k_f = k_inf Pr/(1 + Pr) F, log10 F = log10 Fc / (1 + f1^2),
      // f1 = (log10 Pr + c) / (n' - 0.14 (log10 Pr + c)), c = -0.4 - 0.67 log10 Fc,
      // n' = 0.75 - 1.27 log10 Fc, Fc = (1-a) e^{-T/T***} + a e^{-T/T*} + e^{-T**/T}.
      const double* tp = t.troe + 8 * (t.rrow[r] >> 16);
      const double lnk0 = fma(tp[1], lnT, tp[0]) - tp[2] * invT;
      double Pr = exp(lnk0 - lnkinf) * M;
      Pr = fmax(Pr, 1e-300);
      const double e3 = exp(-T * tp[4]), e1 = exp(-T * tp[5]), e2 = exp(-tp[6] * invT);
      const double Fc = fma(1.0 - tp[3], e3, fma(tp[3], e1, e2));
      const double logFc = log10(Fc);
      const double c = fma(-0.67, logFc, -0.4);
      const double nn = fma(-1.27, logFc, 0.75);
      const double u = log10(Pr) + c;
      const double den = fma(-0.14, u, nn);
      const double invden = 1.0 / den;
      const double f1 = u * invden;
      const double g1 = fma(f1, f1, 1.0);
      const double invg = 1.0 / g1;
      const double logF = logFc * invg;
      const double invPr1 = 1.0 / (1.0 + Pr);
      kf = kf * (Pr * invPr1) * exp(logF * kLn10);
      if (JAC) {
        const double dlnk0_dT = fma(tp[2], invT, tp[1]) * invT;
        const double dlnPr_dT = dlnk0_dT - dlnkf_dT;
        const double dFc_dT = -(1.0 - tp[3]) * tp[4] * e3 - tp[3] * tp[5] * e1 + tp[6] * invT * invT * e2;
        const double df1_du = nn * invden * invden;
        const double df1_dnn = -u * invden * invden;
        const double dlogF_df1 = -logFc * 2.0 * f1 * invg * invg;
        const double dlogF_dx = dlogF_df1 * df1_du;
        const double dlogF_dlogFc = invg + dlogF_df1 * (df1_du * -0.67 + df1_dnn * -1.27);
        // d ln F / dT = ln10 (dlogF/dx dx/dT + dlogF/dlogFc dlogFc/dT), x = log10 Pr
        const double dlnF_dT = fma(dlogF_dx, dlnPr_dT, dlogF_dlogFc * dFc_dT / Fc);
        dlnkf_dT = dlnkf_dT + dlnPr_dT * invPr1 + dlnF_dT;
        dlnkf_dM = (invPr1 + dlogF_dx) / M;
      }
    }
    const double kr = kf * exp(-lnKc);
    const double fwd = w.C[i0] * w.C[i1] * w.C[i2];
    const double rev = w.C[j0] * w.C[j1] * w.C[j2];
    const double base = fma(kf, fwd, -kr * rev);
    const double wM = (type == 1) ? M : 1.0;
    w.q[r] = wM * base;
    if (JAC) {
      const double snh = (w.hh[j0] + w.hh[j1] + w.hh[j2]) - (w.hh[i0] + w.hh[i1] + w.hh[i2]);
      const double dlnKc_dT = (snh - t.nu[dn]) * invT;
      w.kfw[r] = wM * kf;
      w.krw[r] = wM * kr;
      w.dqdT[r] = wM * fma(kf * dlnkf_dT, fwd, -kr * (dlnkf_dT - dlnKc_dT) * rev);
      w.tbs[r] = (type == 1) ? base : ((type == 2) ? dlnkf_dM * base : 0.0);
    }
  }
  __syncwarp();
  double qp = 0.0, cpp = 0.0;
  for (int k = lane; k < Ns; k += 32) {
    double acc = 0.0, accT = 0.0;
    for (int e = t.wptr[k]; e < t.wptr[k + 1]; ++e) {
      const int v = t.went[e];
      const double nuv = t.nu[v >> 16];
      acc = fma(nuv, w.q[v & 0xffff], acc);
      if (JAC) accT = fma(nuv, w.dqdT[v & 0xffff], accT);
    }
    w.wd[k] = acc;
    if (JAC) w.DT[k] = accT;
    qp = fma(w.hh[k], acc, qp);
    cpp = fma(Z[k] * t.invW[k], w.cp[k], cpp);
  }
  s.T = T; s.invT = invT; s.lnT = lnT; s.S = S; s.rho = rho; s.invrho = invrho; s.Ctot = Ctot;
  s.Q = warp_sum(qp);
  s.cpm = warp_sum(cpp);
  __syncwarp();
}

// f^F into f[0..n): f_k = wdot_k W_k / rho, f_T = -T Q / (rho cpm).
__device__ __forceinline__ void chem_rhs_out(const Tab& t, const WS& w, const Scal& s, double* f, int lane) {
  const int Ns = t.Ns;
  for (int k = lane; k < Ns; k += 32) f[k] = w.wd[k] * t.W[k] * s.invrho;
  if (lane == 0) f[Ns] = -s.T * s.Q * s.invrho / s.cpm;
  __syncwarp();
}

// Analytic Jacobian into the n x n matrix J (leading dimension ld) after
// chem_eval<true> at the same state Z.  Columns of D = nu dq/dC are owned by lanes
// (no write conflicts); then the chain rule through C(Y, T) and rho(Y, T).
__device__ __forceinline__ void chem_jac(const Tab& t, const WS& w, const double* Z, const Scal& s, double* J, int lane) {
  const int Ns = t.Ns, n = t.n, ld = w.ld, nsv = t.nsv;
  for (int l = lane; l < Ns; l += 32) {
    for (int k = 0; k < Ns; ++k) J[k * ld + l] = 0.0;
    for (int e = t.cptr[l]; e < t.cptr[l + 1]; ++e) {
      const uint64_t ce = t.cent[e];
      const int r = ce & 0xffff;
      const int mf = (ce >> 16) & 0xf, mr = (ce >> 20) & 0xf;
      const int o1 = (ce >> 24) & 0xff, o2 = (ce >> 32) & 0xff, o3 = (ce >> 40) & 0xff, o4 = (ce >> 48) & 0xff;
      const double dq = fma(w.kfw[r] * t.nu[mf], w.C[o1] * w.C[o2], -w.krw[r] * t.nu[mr] * (w.C[o3] * w.C[o4]));
      const uint64_t s0 = t.rsp[2 * r], s1 = t.rsp[2 * r + 1];
      const int cnt = (int)((s0 >> 48) & 0xff);
      for (int j = 0; j < cnt; ++j) {
        const int k = (s0 >> (8 * j)) & 0xff;
        const int nuv = (int)(int8_t)((s1 >> (8 * j)) & 0xff);
        J[k * ld + l] = fma(t.nu[nuv], dq, J[k * ld + l]);
      }
    }
    for (int i = 0; i < t.n_tb; ++i) {
      const int r = t.tbl[i];
      const int row = t.rrow[r] & 0xffff;
      const double sc = t.effd[row * nsv + l] * w.tbs[r];
      const uint64_t s0 = t.rsp[2 * r], s1 = t.rsp[2 * r + 1];
      const int cnt = (int)((s0 >> 48) & 0xff);
      for (int j = 0; j < cnt; ++j) {
        const int k = (s0 >> (8 * j)) & 0xff;
        const int nuv = (int)(int8_t)((s1 >> (8 * j)) & 0xff);
        J[k * ld + l] = fma(t.nu[nuv], sc, J[k * ld + l]);
      }
    }
  }
  __syncwarp();
  // DC_k = sum_l D_kl C_l ; aux_j = sum_k h/RT_k D_kj
  double hq = 0.0, dqt = 0.0, dcpm = 0.0;
  const double T = s.T, invT = s.invT;
  for (int k = lane; k < Ns; k += 32) {
    double acc = 0.0, col = 0.0;
    for (int l = 0; l < Ns; ++l) {
      acc = fma(J[k * ld + l], w.C[l], acc);
      col = fma(w.hh[l], J[l * ld + k], col);
    }
    w.DC[k] = acc;
    w.aux[k] = col;
    hq = fma(w.hh[k], acc, hq);
    dqt += fma((w.cp[k] - w.hh[k]) * invT, w.wd[k], w.hh[k] * fma(-acc, invT, w.DT[k]));
    const double dcp = fma(fma(fma(t.dcp[3 * nsv + k], T, t.dcp[2 * nsv + k]), T, t.dcp[nsv + k]), T, t.dcp[k]);
    dcpm = fma(Z[k] * t.invW[k], dcp, dcpm);
  }
  const double HQ = warp_sum(hq);
  const double dQT = warp_sum(dqt);
  const double dCPM = warp_sum(dcpm);
  __syncwarp();
  const double invS = 1.0 / s.S;
  const double inv_rhoS = s.invrho * invS;
  const double Phi = T * s.invrho;
  const double invcpm = 1.0 / s.cpm;
  const double PQc = Phi * s.Q * invcpm;
  // species rows: J_kj = (W_k / W_j)(D_kj - (DC_k - wdot_k)/(rho S)), J_kT = (W_k/rho)(DT_k - (DC_k - wdot_k)/T)
  for (int e = lane; e < Ns * Ns; e += 32) {
    const int k = e / Ns, j = e - k * Ns;
    const double a = (w.DC[k] - w.wd[k]) * inv_rhoS;
    J[k * ld + j] = t.W[k] * t.invW[j] * (J[k * ld + j] - a);
  }
  for (int k = lane; k < Ns; k += 32)
    J[k * ld + Ns] = t.W[k] * s.invrho * fma(-(w.DC[k] - w.wd[k]), invT, w.DT[k]);
  // temperature row
  for (int j = lane; j < Ns; j += 32) {
    const double dQ = s.rho * t.invW[j] * w.aux[j] - invS * t.invW[j] * HQ;
    const double dPhi = Phi * invS * t.invW[j];
    J[Ns * ld + j] = -(dPhi * s.Q * invcpm + Phi * dQ * invcpm - PQc * w.cp[j] * t.invW[j] * invcpm);
  }
  if (lane == 0) J[Ns * ld + Ns] = -(2.0 * PQc * invT + Phi * dQT * invcpm - PQc * dCPM * invcpm);
  __syncwarp();
  (void)n;
}

// M = I - hg J in place.
__device__ __forceinline__ void form_newton_matrix(double* M, int n, int ld, double hg, int lane) {
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e - i * n;
    M[i * ld + j] = ((i == j) ? 1.0 : 0.0) - hg * M[i * ld + j];
  }
  __syncwarp();
}

// ------------------------------------------------------------------ dense LU

// In-place LU with partial pivoting (largest |a|; ties to the lowest row).  The
// pivot search compares the magnitudes' IEEE bit patterns as integers, which
// orders non-negative doubles exactly.  dinv[k] = 1 / U_kk.  Returns 0 or k+1 for
// a zero or non-finite pivot in column k (the factorisation stops there).
template <bool SCALED>
__device__ __forceinline__ int lu_factor_warp(double* A, int n, int ld, int* piv, double* dinv, int lane) {
  for (int k = 0; k < n; ++k) {
    unsigned long long best = 0ull;
    int bi = 0x7fffffff;
    for (int i = k + lane; i < n; i += 32) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(A[i * ld + k]) & 0x7fffffffffffffffull;
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (best == 0ull || best >= 0x7ff0000000000000ull) return k + 1;
    if (lane == 0) piv[k] = bi;
    if (bi != k)
      for (int j = lane; j < n; j += 32) {
        const double a = A[k * ld + j];
        A[k * ld + j] = A[bi * ld + j];
        A[bi * ld + j] = a;
      }
    __syncwarp();
    const double inv = 1.0 / A[k * ld + k];
    if (lane == 0) dinv[k] = inv;
    for (int i = k + 1 + lane; i < n; i += 32) A[i * ld + k] *= inv;
    __syncwarp();
    const int m = n - k - 1;
    for (int e = lane; e < m * m; e += 32) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      A[i * ld + j] = fma(-A[i * ld + k], A[k * ld + j], A[i * ld + j]);
    }
    __syncwarp();
  }
  // SCALED: the strict upper triangle is scaled row by row with 1/U_kk, so the back
  // substitution of every later solve needs no multiplication by the diagonal inverse.
  if (SCALED) {
    for (int e = lane; e < n * n; e += 32) {
      const int i = e / n, j = e - i * n;
      if (j > i) A[i * ld + j] *= dinv[i];
    }
    __syncwarp();
  }
  return 0;
}

// Solve with the factors of lu_factor_warp<SCALED>; b is overwritten by x.  SCALED
// factors hold D^-1 U above the diagonal, unscaled ones U (diagonal inverse in dinv).
template <bool SCALED>
__device__ __forceinline__ void lu_solve_warp(const double* A, int n, int ld, const int* piv, const double* dinv,
                                              double* b, int lane) {
  if (lane == 0)
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncwarp();
  for (int j = 0; j < n - 1; ++j) {
    const double xj = b[j];
    for (int i = j + 1 + lane; i < n; i += 32) b[i] = fma(-A[i * ld + j], xj, b[i]);
    __syncwarp();
  }
  if (SCALED) {
    for (int i = lane; i < n; i += 32) b[i] *= dinv[i];
    __syncwarp();
    for (int j = n - 1; j > 0; --j) {
      const double xj = b[j];
      for (int i = lane; i < j; i += 32) b[i] = fma(-A[i * ld + j], xj, b[i]);
      __syncwarp();
    }
  } else {
    for (int j = n - 1; j >= 0; --j) {
      const double xj = b[j] * dinv[j];
      __syncwarp();
      if (lane == 0) b[j] = xj;
      for (int i = lane; i < j; i += 32) b[i] = fma(-A[i * ld + j], xj, b[i]);
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------ stage kernel

struct StageArgs {
  double* y;
  const double* p;
  const double* phi;
  int32_t* status;
  int32_t* stats;
  int32_t* n_failed;
  const unsigned char* table;
  Layout L;
  int ncell, K, n_sub, ramp, max_newton, nstage, sticky, jac_policy;
  double Hs, hh, rtol, atol_Y, atol_T;
  double A[3][3], c[3], gamma;
};

constexpr int kMaxJacAge = 20;
constexpr double kNewtonSafety = 3e-3;

__device__ __forceinline__ void substep_geometry(int s, int ramp, double hh, double& tau, double& hk) {
  if (ramp > 0) {
    if (s == 0) { tau = 0.0; hk = ldexp(hh, -ramp); return; }
    if (s <= ramp) { tau = ldexp(hh, s - 1 - ramp); hk = tau; return; }
    tau = (double)(s - ramp) * hh;
    hk = hh;
    return;
  }
  tau = (double)s * hh;
  hk = hh;
}

// WRMS norm of the Newton correction d with weights from the updated iterate Z + d.
__device__ __forceinline__ double wrms_update(const double* d, const double* Z, int n, double rtol, double atolY, double atolT,
                              int lane) {
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) {
    const double wgt = fma(rtol, fabs(Z[k] + d[k]), (k == n - 1) ? atolT : atolY);
    const double v = d[k] / wgt;
    acc = fma(v, v, acc);
  }
  return sqrt(warp_sum(acc) / n);
}

// Jacobian at Z, M = I - hg J, LU.  Returns the LU info (0 = ok).
__device__ __forceinline__ int refresh_matrix(const Tab& t, const WS& w, const double* Z, double p, double hg, int lane) {
  Scal s;
  chem_eval<true>(t, w, Z, p, s, lane);
  chem_jac(t, w, Z, s, w.M, lane);
  form_newton_matrix(w.M, t.n, w.ld, hg, lane);
  return lu_factor_warp<true>(w.M, t.n, w.ld, w.piv, w.dinv, lane);
}

__global__ void __launch_bounds__(kMaxWarps * 32) stage_fast_kernel(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table(smem, a.table, a.L.bytes);
  __syncthreads();
  const Tab t(smem, a.L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const WS w(reinterpret_cast<double*>(smem + a.L.bytes) + (size_t)warp * a.L.ws_doubles, a.L);
  const int n = t.n, Ns = t.Ns, S = a.nstage;
  const int total_sub = a.n_sub + (a.ramp > 0 ? a.ramp : 0);
  for (int cell = blockIdx.x * nw + warp; cell < a.ncell; cell += gridDim.x * nw) {
    double* yc = a.y + (size_t)cell * n;
    const double p = a.p[cell];
    int bad = 0;
    for (int k = lane; k < n; k += 32) {
      const double v = yc[k];
      w.y0[k] = v;
      if (!isfinite(v)) bad = 1;
    }
    for (int e = lane; e < a.K * n; e += 32) w.phi[(e / n) * w.nv + (e % n)] = a.phi[(size_t)cell * a.K * n + e];
    __syncwarp();
    bad = __any_sync(0xffffffffu, bad) || !(w.y0[Ns] > 0.0) || !(p > 0.0) || !isfinite(p);
    int status = bad ? MRI_CELL_EINPUT : MRI_CELL_OK;
    int nsub = 0, nnewton = 0, njac = 0;
    double M_hg = 0.0;     // h gamma of the factorised Newton matrix (0: none yet)
    int M_age = 0;         // substeps since its Jacobian was evaluated
    for (int sidx = 0; sidx < total_sub && status == MRI_CELL_OK; ++sidx) {
      double tau, hk;
      substep_geometry(sidx, a.ramp, a.hh, tau, hk);
      const double hg = hk * a.gamma;
      const double inv_hg = 1.0 / hg;
      const bool startup_sub = (a.ramp > 0 && sidx <= a.ramp);
      // MRI_JAC_PER_SUBSTEP: Jacobian + LU at every substep start.  MRI_JAC_LAZY: the
      // factorised matrix carries over while h gamma is unchanged and it is younger
      // than kMaxJacAge substeps; poor contraction refreshes it inside Newton.
      const bool need = (a.jac_policy == MRI_JAC_PER_SUBSTEP) || startup_sub || hg != M_hg ||
                        M_age >= kMaxJacAge;
      if (need) {
        if (refresh_matrix(t, w, w.y0, p, hg, lane) != 0) { status = MRI_CELL_ENEWTON; break; }
        njac++;
        M_hg = hg;
        M_age = 0;
      } else {
        M_age++;
      }
      for (int k = lane; k < n; k += 32) w.Z[k] = w.y0[k];
      __syncwarp();
      for (int i = 0; i < S && status == MRI_CELL_OK; ++i) {
        const double rh = (tau + a.c[i] * hk) / a.Hs;
        for (int k = lane; k < n; k += 32) {
          double rv = 0.0;
          for (int j = a.K - 1; j >= 0; --j) rv = fma(rv, rh, w.phi[j * w.nv + k]);
          w.r[k] = rv;
          double bs = w.y0[k];
          for (int j = 0; j < i; ++j) bs = fma(hk * a.A[i][j], w.F[j][k], bs);
          w.base[k] = bs;   // stage base y_n + h sum_j a_ij F_j
        }
        __syncwarp();
        // Modified Newton: the matrix of the substep start is reused while it
        // contracts.  When an iteration contracts poorly (or leaves the finite
        // range) with a matrix older than the current iterate, the iteration is
        // redone with a fresh Jacobian at the current iterate (a full Newton step;
        // the residual is reused).  Start-up substeps use full Newton throughout.
        // The converged stage value does not depend on the matrix policy.
        const bool startup = startup_sub;
        bool fresh = (i == 0) && need;
        bool conv = false;
        double prev = 0.0;
        for (int it = 0; it < a.max_newton; ++it) {
          Scal s;
          chem_eval<false>(t, w, w.Z, p, s, lane);
          chem_rhs_out(t, w, s, w.f, lane);
          for (int k = lane; k < n; k += 32) {
            const double g = -(w.Z[k] - w.base[k] - hg * (w.f[k] + w.r[k]));
            w.res[k] = g;
            w.d[k] = g;
          }
          __syncwarp();
          if (startup && !fresh) {   // start-up substeps: full Newton, as far from the manifold
            if (refresh_matrix(t, w, w.Z, p, hg, lane) != 0) break;
            njac++;
            fresh = true;
          }
          lu_solve_warp<true>(w.M, n, w.ld, w.piv, w.dinv, w.d, lane);
          double nrm = wrms_update(w.d, w.Z, n, a.rtol, a.atol_Y, a.atol_T, lane);
          // redo with a fresh matrix when the stale one contracts by less than 10x, or
          // when its contraction rate would not reach the tolerance three iterations
          // before max_newton
          bool redo = !fresh && (!isfinite(nrm) || (it > 0 && nrm > 0.1 * prev));
          if (!fresh && !redo && it > 0 && nrm > 1.0) {
            const double rho = nrm / prev;
            double proj = nrm;
            const int left = a.max_newton - 3 - (it + 1);
            for (int j = 0; j < left && proj > 1.0; ++j) proj *= rho;
            redo = proj > 1.0;
          }
          if (redo) {
            if (refresh_matrix(t, w, w.Z, p, hg, lane) != 0) break;
            njac++;
            M_age = 0;
            for (int k = lane; k < n; k += 32) w.d[k] = w.res[k];
            __syncwarp();
            lu_solve_warp<true>(w.M, n, w.ld, w.piv, w.dinv, w.d, lane);
            nrm = wrms_update(w.d, w.Z, n, a.rtol, a.atol_Y, a.atol_T, lane);
          }
          for (int k = lane; k < n; k += 32) w.Z[k] += w.d[k];
          __syncwarp();
          const bool full_step = fresh || redo;
          fresh = false;
          nnewton++;
          if (!isfinite(nrm)) break;
          // A full Newton step converges quadratically: accept WRMS(delta) <= 1.  A step
          // with an older matrix converges linearly with rate rho = nrm / prev; its
          // remaining error is about rho * nrm, which must also be small, so that the
          // accepted iterate matches the exact stage solution far inside the tolerance.
          if (full_step ? (nrm <= 1.0) : (it > 0 && nrm <= 1.0 && nrm * (nrm / prev) <= kNewtonSafety)) {
            conv = true;
            break;
          }
          prev = nrm;
        }
        if (!conv) { status = MRI_CELL_ENEWTON; break; }
        if (i < S - 1) {
          for (int k = lane; k < n; k += 32) w.F[i][k] = (w.Z[k] - w.base[k]) * inv_hg;
          __syncwarp();
        }
      }
      if (status != MRI_CELL_OK) break;
      for (int k = lane; k < n; k += 32) w.y0[k] = w.Z[k];
      __syncwarp();
      nsub++;
    }
    if (status != MRI_CELL_EINPUT)
      for (int k = lane; k < n; k += 32) yc[k] = w.y0[k];
    if (lane == 0) {
      if (a.status && (!a.sticky || status != MRI_CELL_OK)) a.status[cell] = status;
      if (a.stats) {
        int32_t* st = a.stats + 4 * (size_t)cell;
        st[0] += nsub; st[1] += nnewton; st[2] += njac; st[3] += (status != MRI_CELL_OK);
      }
      if (a.n_failed && status != MRI_CELL_OK) atomicAdd(a.n_failed, 1);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ per-kernel entry kernels

__global__ void __launch_bounds__(kMaxWarps * 32) rhs_kernel(const double* y, const double* p, int ncell,
                                                              double* f, const unsigned char* table, Layout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table(smem, table, L.bytes);
  __syncthreads();
  const Tab t(smem, L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const WS w(reinterpret_cast<double*>(smem + L.bytes) + (size_t)warp * L.ws_doubles, L);
  for (int cell = blockIdx.x * nw + warp; cell < ncell; cell += gridDim.x * nw) {
    for (int k = lane; k < t.n; k += 32) w.Z[k] = y[(size_t)cell * t.n + k];
    __syncwarp();
    Scal s;
    chem_eval<false>(t, w, w.Z, p[cell], s, lane);
    chem_rhs_out(t, w, s, w.f, lane);
    for (int k = lane; k < t.n; k += 32) f[(size_t)cell * t.n + k] = w.f[k];
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kMaxWarps * 32) jac_kernel(const double* y, const double* p, int ncell,
                                                              double* J, const unsigned char* table, Layout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table(smem, table, L.bytes);
  __syncthreads();
  const Tab t(smem, L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const WS w(reinterpret_cast<double*>(smem + L.bytes) + (size_t)warp * L.ws_doubles, L);
  const int n = t.n;
  for (int cell = blockIdx.x * nw + warp; cell < ncell; cell += gridDim.x * nw) {
    for (int k = lane; k < n; k += 32) w.Z[k] = y[(size_t)cell * n + k];
    __syncwarp();
    Scal s;
    chem_eval<true>(t, w, w.Z, p[cell], s, lane);
    chem_jac(t, w, w.Z, s, w.M, lane);
    for (int e = lane; e < n * n; e += 32) J[(size_t)cell * n * n + e] = w.M[(e / n) * w.ld + e % n];
    __syncwarp();
  }
}

__global__ void lu_kernel(double* A, double* b, int n, int ld, int nbatch, int32_t* info) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = round_up(n * ld, 2) + 2 * round_up(n, 2) + n;
  double* Ms = reinterpret_cast<double*>(smem) + (size_t)warp * per;
  double* bs = Ms + round_up(n * ld, 2);
  double* dv = bs + round_up(n, 2);
  int* pv = reinterpret_cast<int*>(dv + round_up(n, 2));
  for (int sys = blockIdx.x * nw + warp; sys < nbatch; sys += gridDim.x * nw) {
    for (int e = lane; e < n * n; e += 32) Ms[(e / n) * ld + e % n] = A[(size_t)sys * n * n + e];
    for (int k = lane; k < n; k += 32) bs[k] = b[(size_t)sys * n + k];
    __syncwarp();
    const int rc = lu_factor_warp<false>(Ms, n, ld, pv, dv, lane);
    if (rc == 0) lu_solve_warp<false>(Ms, n, ld, pv, dv, bs, lane);
    for (int e = lane; e < n * n; e += 32) A[(size_t)sys * n * n + e] = Ms[(e / n) * ld + e % n];
    for (int k = lane; k < n; k += 32) b[(size_t)sys * n + k] = bs[k];
    if (lane == 0 && info) info[sys] = rc;
    __syncwarp();
  }
}

// ------------------------------------------------------------------ host side

int device_sm_count() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

int device_smem_limit() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v > 0 ? v : 48 * 1024;
}

// Warps per CTA and grid for a warp-per-cell kernel with `per_warp` bytes of workspace.
static bool plan_launch(const Layout& L, int ncell, int& warps, int& blocks, size_t& smem) {
  const int limit = device_smem_limit();
  const size_t per_warp = (size_t)L.ws_doubles * 8;
  int wmax = (int)((limit - L.bytes) / (long long)per_warp);
  if (wmax < 1) return false;
  if (wmax > kMaxWarps) wmax = kMaxWarps;
  const int sms = device_sm_count();
  int want = (ncell + sms - 1) / sms;
  warps = want < 1 ? 1 : (want > wmax ? wmax : want);
  blocks = (ncell + warps - 1) / warps;
  if (blocks > sms) blocks = sms;
  if (blocks < 1) blocks = 1;
  smem = (size_t)L.bytes + (size_t)warps * per_warp;
  return true;
}

static void sdirk_table(int method, StageArgs& a) {
  for (int i = 0; i < 3; ++i) {
    a.c[i] = 0.0;
    for (int j = 0; j < 3; ++j) a.A[i][j] = 0.0;
  }
  if (method == MRI_SDIRK2) {
    const double g = 0.29289321881345247559915563789515;   // 1 - 1/sqrt(2)
    a.gamma = g;
    a.A[0][0] = g;
    a.A[1][0] = 1.0 - g; a.A[1][1] = g;
    a.c[0] = g; a.c[1] = 1.0;
    a.nstage = 2;
  } else {
    // L-stable root of g^3 - 3 g^2 + 3/2 g - 1/6 = 0
    const double g = 0.43586652150845899941601945119356;
    a.gamma = g;
    a.A[0][0] = g;
    a.A[1][0] = 0.5 * (1.0 - g); a.A[1][1] = g;
    a.A[2][0] = 0.25 * (-6.0 * g * g + 16.0 * g - 1.0);
    a.A[2][1] = 0.25 * (6.0 * g * g - 20.0 * g + 5.0);
    a.A[2][2] = g;
    a.c[0] = g; a.c[1] = 0.5 * (1.0 + g); a.c[2] = 1.0;
    a.nstage = 3;
  }
}

int launch_stage_fast(double* y, const double* p, int ncell, const double* phi, int K, double Hs, double h,
                      const Mech& m, const mri_fast_opts& o, int ramp, int32_t* status, int32_t* stats,
                      int32_t* n_failed, cudaStream_t st, bool sticky) {
  if (ncell == 0) return MRI_OK;
  StageArgs a{};
  a.sticky = sticky ? 1 : 0;
  a.y = y; a.p = p; a.phi = phi; a.status = status; a.stats = stats; a.n_failed = n_failed;
  a.table = static_cast<const unsigned char*>(m.d_table);
  a.L = m.L;
  a.ncell = ncell; a.K = K;
  double r = Hs / h;
  double nsub = std::ceil(r * (1.0 - 1e-12));
  if (!(nsub >= 1.0)) nsub = 1.0;
  if (nsub > 1e7) return MRI_EINVAL;
  a.n_sub = (int)nsub;
  a.hh = Hs / a.n_sub;
  a.Hs = Hs;
  a.ramp = ramp;
  a.max_newton = o.max_newton;
  a.jac_policy = o.jac_policy;
  a.rtol = o.newton_rtol; a.atol_Y = o.newton_atol_Y; a.atol_T = o.newton_atol_T;
  sdirk_table(o.method, a);
  int warps, blocks;
  size_t smem;
  if (!plan_launch(m.L, ncell, warps, blocks, smem)) return MRI_EINVAL;
  if (cudaFuncSetAttribute(stage_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MRI_ECUDA;
  stage_fast_kernel<<<blocks, warps * 32, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

}  // namespace mri

// ------------------------------------------------------------------ C ABI

namespace mri {

bool fast_opts_ok(const mri_fast_opts* o) {
  return o && (o->method == MRI_SDIRK2 || o->method == MRI_SDIRK3) && o->newton_rtol > 0 &&
         std::isfinite(o->newton_rtol) && o->newton_atol_Y >= 0 && o->newton_atol_T >= 0 &&
         std::isfinite(o->newton_atol_Y) && std::isfinite(o->newton_atol_T) && o->max_newton >= 1 &&
         o->max_newton <= 100 && (o->jac_policy == MRI_JAC_PER_SUBSTEP || o->jac_policy == MRI_JAC_LAZY) &&
         o->precision == MRI_PREC_FP64 &&
         o->ramp >= 0 && o->ramp <= 40;
}

int mri_stage_fast_checked(double* y, const double* p, int ncell, const double* phi, int K, double Hstage,
                           double h, const Mech& m, const mri_fast_opts& o, int32_t* cell_status,
                           int32_t* cell_stats, int32_t* n_failed, cudaStream_t st, bool sticky) {
  if (!fast_opts_ok(&o) || ncell < 0 || K < 0 || K > kMaxK) return MRI_EINVAL;
  if (!(Hstage > 0) || !(h > 0) || !std::isfinite(Hstage) || !std::isfinite(h)) return MRI_EINVAL;
  if (ncell > 0 && (!y || !p || (K > 0 && !phi))) return MRI_EINVAL;
  return launch_stage_fast(y, p, ncell, phi, K, Hstage, h, m, o, o.ramp, cell_status, cell_stats, n_failed, st,
                           sticky);
}

}  // namespace mri

using mri::Mech;

extern "C" void mri_fast_opts_default(mri_fast_opts* o) {
  if (!o) return;
  o->method = MRI_SDIRK3;
  o->newton_rtol = 1e-10;
  o->newton_atol_Y = 1e-20;
  o->newton_atol_T = 1e-10;
  o->max_newton = 10;
  o->jac_policy = MRI_JAC_PER_SUBSTEP;
  o->precision = MRI_PREC_FP64;
  o->ramp = 0;
}

extern "C" int mri_stage_fast(double* y, const double* p, int ncell, const double* phi, int K, double t0,
                              double Hstage, double h, const mri_mech* mech, const mri_fast_opts* opts,
                              int32_t* cell_status, int32_t* cell_stats, int32_t* n_failed, void* stream) {
  (void)t0;   // the chemistry is autonomous; the forcing uses time relative to the stage start
  if (!mech || !mri::fast_opts_ok(opts) || ncell < 0 || K < 0 || K > mri::kMaxK) return MRI_EINVAL;
  if (!(Hstage > 0) || !(h > 0) || !std::isfinite(Hstage) || !std::isfinite(h)) return MRI_EINVAL;
  return mri::mri_stage_fast_checked(y, p, ncell, phi, K, Hstage, h, *reinterpret_cast<const Mech*>(mech), *opts,
                                     cell_status, cell_stats, n_failed, static_cast<cudaStream_t>(stream), false);
}

extern "C" int mri_fast_rhs(const double* y, const double* p, int ncell, const mri_mech* mech, double* f,
                            void* stream) {
  if (!mech || ncell < 0 || (ncell > 0 && (!y || !p || !f))) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  const Mech* m = reinterpret_cast<const Mech*>(mech);
  int warps, blocks;
  size_t smem;
  if (!mri::plan_launch(m->L, ncell, warps, blocks, smem)) return MRI_EINVAL;
  if (cudaFuncSetAttribute(mri::rhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MRI_ECUDA;
  mri::rhs_kernel<<<blocks, warps * 32, smem, static_cast<cudaStream_t>(stream)>>>(
      y, p, ncell, f, static_cast<const unsigned char*>(m->d_table), m->L);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_fast_jac(const double* y, const double* p, int ncell, const mri_mech* mech, double* J,
                            void* stream) {
  if (!mech || ncell < 0 || (ncell > 0 && (!y || !p || !J))) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  const Mech* m = reinterpret_cast<const Mech*>(mech);
  int warps, blocks;
  size_t smem;
  if (!mri::plan_launch(m->L, ncell, warps, blocks, smem)) return MRI_EINVAL;
  if (cudaFuncSetAttribute(mri::jac_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MRI_ECUDA;
  mri::jac_kernel<<<blocks, warps * 32, smem, static_cast<cudaStream_t>(stream)>>>(
      y, p, ncell, J, static_cast<const unsigned char*>(m->d_table), m->L);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_lu_solve_batched(double* A, double* b, int n, int nbatch, int32_t* info, void* stream) {
  if (n < 1 || n > 128 || nbatch < 0 || (nbatch > 0 && (!A || !b))) return MRI_EINVAL;
  if (nbatch == 0) return MRI_OK;
  const int ld = (n % 2 == 1) ? n : n + 1;
  const size_t per = ((size_t)mri::round_up(n * ld, 2) + 2 * mri::round_up(n, 2) + n) * 8;
  const int limit = mri::device_smem_limit();
  int warps = (int)(limit / per);
  if (warps < 1) return MRI_EINVAL;
  if (warps > 8) warps = 8;
  int blocks = (nbatch + warps - 1) / warps;
  const int cap = mri::device_sm_count() * 4;
  if (blocks > cap) blocks = cap;
  const size_t smem = per * warps;
  if (cudaFuncSetAttribute(mri::lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MRI_ECUDA;
  mri::lu_kernel<<<blocks, warps * 32, smem, static_cast<cudaStream_t>(stream)>>>(A, b, n, ld, nbatch, info);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}
