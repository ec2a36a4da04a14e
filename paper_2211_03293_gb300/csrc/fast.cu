// The fast-partition hot path: chemistry right-hand side, analytic Jacobian,
// warp-cooperative dense LU and the SDIRK / Newton substep driver.
//
// Organisation: a persistent grid (one CTA per SM) whose warps take cells from a
// device work queue; a warp owns one grid cell for a whole MRI stage.  The
// mechanism table lives in shared memory (one copy per CTA); each warp has a
// private shared-memory workspace with the cell's n x n Newton matrix and the
// vectors of the stage.  Lanes split reactions (rates), species (sums over
// reactions), Jacobian columns (assembly) and matrix rows/entries (LU).  The state,
// residual and rates are FP64; the Newton matrix, its LU and the triangular solves
// are FP64 or, in the mixed-precision form (PREC32), FP32.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <utility>
#include <vector>

#include "fastmath.cuh"
#include "internal.cuh"

namespace mri {

// ------------------------------------------------------------------ views

struct Tab {
  const double *cp, *hh, *ss, *h5, *s6, *dcp, *W, *invW, *lnA, *b, *Ta, *eval, *troe, *nu, *exp2t, *logt, *tcv;
  const float *nu32, *W32, *invW32, *dcp32, *tcv32;
  const uint64_t *rxn, *cent, *rsp;
  const int32_t *rrow, *eptr, *eidx, *cptr, *tbl, *trx, *tcptr, *tcr, *gent, *gsptr, *gslot;
  int Ns, R, n, nsv, n_tb, n_troe, g_chunk, n_went;
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
    eval = reinterpret_cast<const double*>(s + L.o_eval);
    troe = reinterpret_cast<const double*>(s + L.o_troe);
    nu = reinterpret_cast<const double*>(s + L.o_nu) + 3;   // nu[v] for v in -3..4
    exp2t = reinterpret_cast<const double*>(s + L.o_exp2);
    logt = reinterpret_cast<const double*>(s + L.o_logt);
    nu32 = reinterpret_cast<const float*>(s + L.o_nu32) + 3;
    W32 = reinterpret_cast<const float*>(s + L.o_W32);
    invW32 = reinterpret_cast<const float*>(s + L.o_invW32);
    dcp32 = reinterpret_cast<const float*>(s + L.o_dcp32);
    rxn = reinterpret_cast<const uint64_t*>(s + L.o_rxn);
    cent = reinterpret_cast<const uint64_t*>(s + L.o_cent);
    rsp = reinterpret_cast<const uint64_t*>(s + L.o_rsp);
    rrow = reinterpret_cast<const int32_t*>(s + L.o_rrow);
    eptr = reinterpret_cast<const int32_t*>(s + L.o_eptr);
    eidx = reinterpret_cast<const int32_t*>(s + L.o_eidx);
    cptr = reinterpret_cast<const int32_t*>(s + L.o_cptr);
    tbl = reinterpret_cast<const int32_t*>(s + L.o_tbl);
    trx = reinterpret_cast<const int32_t*>(s + L.o_trx);
    tcptr = reinterpret_cast<const int32_t*>(s + L.o_tcptr);
    gent = reinterpret_cast<const int32_t*>(s + L.o_gent);
    gsptr = reinterpret_cast<const int32_t*>(s + L.o_gsptr);
    gslot = reinterpret_cast<const int32_t*>(s + L.o_gslot);
    tcr = reinterpret_cast<const int32_t*>(s + L.o_tcr);
    tcv = reinterpret_cast<const double*>(s + L.o_tcv);
    tcv32 = reinterpret_cast<const float*>(s + L.o_tcv32);
    Ns = L.Ns; R = L.R; n = L.n; nsv = L.nsv; n_tb = L.n_tb; n_troe = L.n_troe;
    g_chunk = L.g_chunk; n_went = L.n_went;
  }
};

struct WS {
  double *M, *y0, *Z, *d, *res, *F0, *F1, *Fl, *r, *f, *base, *phi, *C, *hh, *cp, *wd, *DT, *DC, *aux, *dinv;
  double *E, *Einv, *c0p, *tro, *tbk;
  int* piv;
  double *q, *kfw, *krw, *dqdT, *tbs;
  // mixed-precision form: FP32 Newton matrix, its diagonal inverse and FP32 copies
  float *M32, *dinv32, *d32, *C32, *hh32, *cp32, *wd32, *DT32, *DC32, *aux32, *tbk32, *kfw32, *krw32, *tbs32;
  int ld, nv;
  __device__ __forceinline__ double* F(int j) const { return j == 0 ? F0 : F1; }
  __device__ WS(double* base, const Layout& L, bool prec32, int K, bool matrix = true) {
    WsOffsets o = ws_offsets(L, prec32, K, matrix);
    M = base + o.M; y0 = base + o.y0; Z = base + o.Z; d = base + o.d;
    F0 = base + o.F0; F1 = base + o.F1; Fl = base + o.Fl; r = base + o.r; phi = base + o.phi;
    f = (o.f >= 0) ? base + o.f : nullptr;
    this->base = base + o.base;
    res = base + o.res;
    C = base + o.C; hh = base + o.hh; cp = base + o.cp; wd = base + o.wd;
    DT = base + o.DT; DC = base + o.DC; aux = base + o.aux; dinv = base + o.dinv;
    E = base + o.E; Einv = base + o.Einv; c0p = base + o.c0p; tro = base + o.tro; tbk = base + o.tbk;
    piv = reinterpret_cast<int*>(base + o.piv);
    q = base + o.q; kfw = base + o.kfw; krw = base + o.krw; dqdT = base + o.dqdT; tbs = base + o.tbs;
    float* fb = reinterpret_cast<float*>(base + o.f32);
    const F32Offsets g32 = f32_offsets(L, o.r32 != 0);
    M32 = reinterpret_cast<float*>(base + o.M);
    dinv32 = fb + g32.dinv;
    C32 = fb + g32.C; hh32 = fb + g32.hh; cp32 = fb + g32.cp; wd32 = fb + g32.wd; DT32 = fb + g32.DT;
    tbk32 = fb + g32.tbk;
    if (o.r32) {
      // in dead FP64 scratch: the reaction copies in the rates and the falloff scratch
      // (dead when the copies are made), DC and the column sums in E and 1/E (as in the
      // FP64 form), the correction in the rates again (no rates are live in a solve)
      kfw32 = reinterpret_cast<float*>(base + o.q);
      krw32 = kfw32 + L.rv;
      tbs32 = reinterpret_cast<float*>(base + o.tro);
      DC32 = reinterpret_cast<float*>(base + o.E);
      aux32 = DC32 + round_up(L.nsv, 4);
      d32 = reinterpret_cast<float*>(base + o.q);
    } else {
      kfw32 = fb + g32.kfw; krw32 = fb + g32.krw; tbs32 = fb + g32.tbs;
      DC32 = fb + g32.DC; aux32 = fb + g32.aux; d32 = fb + g32.d;
    }
    ld = L.ld;
    nv = round_up(L.n + 1, 2);
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
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
  double T, invT, lnT, S, invS, rho, invrho, Ctot, cpm, invcpm, Q;
};

// dst[k] = sum_r nu_kr src[r] for every species, balanced over the lanes: lane l
// sums entries [l L, (l+1) L) of the species-major (species, reaction, nu) list,
// ending every run of one species in a partial-sum slot (the slots reuse the
// falloff scratch, free after the reaction pass); then each species adds its slots
// in a fixed order, so the sums are deterministic.
__device__ __forceinline__ void gather_species(const Tab& t, const WS& w, const double* src, double* dst, int lane) {
  double* P = w.tro;
  double acc = 0.0;
  const int e1 = min((lane + 1) * t.g_chunk, t.n_went);
  for (int e = lane * t.g_chunk; e < e1; ++e) {
    const int v = t.gent[e];
    acc = fma(t.nu[((v >> 10) & 0xf) - 8], src[v & 0x3ff], acc);
    if ((v >> 22) & 1) {
      P[(v >> 14) & 0xff] = acc;
      acc = 0.0;
    }
  }
  __syncwarp();
  for (int k = lane; k < t.Ns; k += 32) {
    double sum = 0.0;
    for (int j = t.gsptr[k]; j < t.gsptr[k + 1]; ++j) sum += P[t.gslot[j]];
    dst[k] = sum;
  }
  __syncwarp();
}

struct RxnOut {
  double q, kfw, krw, dqdT, tbs;
};

// Rate of progress of reaction r (and with JAC its Jacobian pieces) from the species
// factors of chem_eval: k_f = k_inf (times the falloff factor Pr/(1+Pr) F, whose ln F
// joins the exponent of k_inf), 1/K_c as a product of species factors,
// q = [M] (k_f prod C^nu' - k_r prod C^nu'').  PLAIN: the caller guarantees a
// reaction without third body or falloff ([M] = 1), and the code has no branches on
// the reaction type (the same values as the general code).
template <bool JAC, bool PLAIN = false>
__device__ __forceinline__ void rxn_eval(const Tab& t, const WS& w, int r, double lnT, double invT, double Ctot,
                                         RxnOut& o) {
  const uint64_t rec = t.rxn[r];
  const int i0 = rec & 0xff, i1 = (rec >> 8) & 0xff, i2 = (rec >> 16) & 0xff;
  const int j0 = (rec >> 24) & 0xff, j1 = (rec >> 32) & 0xff, j2 = (rec >> 40) & 0xff;
  const int dn = (int)(int8_t)((rec >> 48) & 0xff);
  const int type = PLAIN ? 0 : (int)(rec >> 56);
  const int tr = PLAIN ? 0 : t.rrow[r] >> 16;      // falloff row (type 2)
  double lnkf = fma(t.b[r], lnT, t.lnA[r]) - t.Ta[r] * invT;
  if (type == 2) lnkf += w.tro[kTroeSlots * tr + 6];      // ln F
  double kf = exp_tab(lnkf, t.exp2t);
  if (type == 2) kf *= w.tro[kTroeSlots * tr + 9];        // Pr / (1 + Pr)
  double M = 1.0;
  if (type == 1) {
    const int row = t.rrow[r] & 0xffff;
    M = Ctot;
    for (int e = t.eptr[row]; e < t.eptr[row + 1]; ++e) M = fma(t.eval[e], w.C[t.eidx[e]], M);
  }
  const double fwd = w.C[i0] * w.C[i1] * w.C[i2];
  // 1 / K_c = prod_reactants E * prod_products 1/E * (p_atm/RT)^(-dn).  Without the
  // Jacobian the product factors come premultiplied by their concentrations
  // (CE_k = C_k / E_k, in the 1/E array), so k_r prod C^nu'' = k_f Er prod CE.
  const double Er = (w.E[i0] * w.E[i1]) * (w.E[i2] * w.c0p[dn + 2]);
  if (!JAC) {
    const double q = kf * fma(-Er, w.Einv[j0] * w.Einv[j1] * w.Einv[j2], fwd);
    o.q = PLAIN ? q : M * q;
    return;
  }
  const double kr = kf * (Er * (w.Einv[j0] * w.Einv[j1] * w.Einv[j2]));
  const double rev = w.C[j0] * w.C[j1] * w.C[j2];
  const double base = fma(kf, fwd, -kr * rev);
  o.q = PLAIN ? base : M * base;
  {
    double dlnkf_dT = fma(t.Ta[r], invT, t.b[r]) * invT;
    if (type == 2) dlnkf_dT += w.tro[kTroeSlots * tr + 10];
    const double snh = (w.hh[j0] + w.hh[j1] + w.hh[j2]) - (w.hh[i0] + w.hh[i1] + w.hh[i2]);
    const double dlnKc_dT = (snh - t.nu[dn]) * invT;
    const double dq = fma(kf * dlnkf_dT, fwd, -kr * (dlnkf_dT - dlnKc_dT) * rev);
    o.kfw = PLAIN ? kf : M * kf;
    o.krw = PLAIN ? kr : M * kr;
    o.dqdT = PLAIN ? dq : M * dq;
    o.tbs = (type == 1) ? base : ((type == 2) ? w.tro[kTroeSlots * tr + 11] * base : 0.0);
  }
}

// Species concentrations, NASA-7 thermo, rates of progress, production rates and
// f^F at state Z (Y_1..Y_Ns, T).  With JAC also the per-reaction pieces of the
// Jacobian: [M]-weighted k_f, k_r, d q / d T, the third-body scale and
// sum_r nu dq/dT per species.
//
// Transcendentals are spread so that every lane of a pass has one to evaluate:
//  * 1/K_c of every reaction is a product of per-species factors
//    E_k = exp(-g_k/RT) (reactants) and 1/E_k (products) times (p_atm/RT)^(-dn),
//    so a reaction needs one exponential (k_f) instead of two;
//  * the falloff (Troe) quantities are evaluated task-parallel before the
//    reaction pass: 4 exponentials per falloff reaction in one pass, then the two
//    log10, then the broadening factor, each falloff reaction on its own lane.
template <bool JAC>
__device__ __forceinline__ void chem_eval(const Tab& t, const WS& w, const double* Z, double p, Scal& s, int lane) {
  const int Ns = t.Ns, R = t.R, nsv = t.nsv, NT = t.n_troe;
  const double T = Z[Ns];
  double part = 0.0;
  for (int k = lane; k < Ns; k += 32) part = fma(Z[k], t.invW[k], part);
  const double S = warp_sum(part);
  // 1/T, 1/S and 1/p in one division: lane 0 inverts T, lane 1 S, lane 2 p
  const double dv = 1.0 / ((lane == 0) ? T : (lane == 1) ? S : p);
  const double invT = __shfl_sync(0xffffffffu, dv, 0);
  const double invS = __shfl_sync(0xffffffffu, dv, 1);
  const double invp = __shfl_sync(0xffffffffu, dv, 2);
  const double lnT = log_tab(T, t.logt);
  const double rho = (p * (1.0 / kRu)) * (invT * invS);
  const double invrho = (kRu * T) * (S * invp);
  double cpp = 0.0;
  for (int k = lane; k < Ns; k += 32) {
    const double zw = Z[k] * t.invW[k];
    const double c = rho * zw;
    w.C[k] = c;
    double cpv = fma(fma(fma(fma(t.cp[4 * nsv + k], T, t.cp[3 * nsv + k]), T, t.cp[2 * nsv + k]), T,
                         t.cp[nsv + k]), T, t.cp[k]);
    double hv = fma(fma(fma(fma(t.hh[4 * nsv + k], T, t.hh[3 * nsv + k]), T, t.hh[2 * nsv + k]), T,
                        t.hh[nsv + k]), T, t.hh[k]) + t.h5[k] * invT;
    double sv = fma(fma(fma(fma(t.ss[4 * nsv + k], T, t.ss[3 * nsv + k]), T, t.ss[2 * nsv + k]), T,
                        t.ss[nsv + k]), T, fma(t.ss[k], lnT, t.s6[k]));
    const double g = hv - sv;
    double e, einv;
    exp_pair(-g, t.exp2t, e, einv);
    cpp = fma(zw, cpv, cpp);
    w.cp[k] = cpv;
    w.hh[k] = hv;
    w.E[k] = e;
    w.Einv[k] = JAC ? einv : c * einv;   // 1/E for the Jacobian's k_r, else C/E
  }
  if (lane == 0) { w.C[Ns] = 1.0; w.hh[Ns] = 0.0; w.E[Ns] = 1.0; w.Einv[Ns] = 1.0; }
  if (lane < 5) {
    // (p_atm / (R T))^(-dn) for dn = -2..2 at index dn + 2
    const double C0 = (kPatm / kRu) * invT, iC0 = (kRu / kPatm) * T;
    const double v = (lane == 0) ? C0 * C0 : (lane == 1) ? C0 : (lane == 2) ? 1.0 : (lane == 3) ? iC0 : iC0 * iC0;
    w.c0p[lane] = v;
  }
  // sum_k C_k = rho sum_k Y_k / W_k = p / (R T): no reduction needed
  const double Ctot = (p * (1.0 / kRu)) * invT;
  const double cpm = warp_sum(cpp);
  __syncwarp();
  // falloff, phase 1: exp(ln k0 - ln k_inf), e^{-T/T***}, e^{-T/T*}, e^{-T**/T}
  for (int e = lane; e < 4 * NT; e += 32) {
    const int tr = e >> 2, kind = e & 3;
    const int r = t.trx[tr];
    const double* tp = t.troe + 8 * tr;
    const double lnkinf = fma(t.b[r], lnT, t.lnA[r]) - t.Ta[r] * invT;
    const double lnk0 = fma(tp[1], lnT, tp[0]) - tp[2] * invT;
    const double arg = (kind == 0) ? lnk0 - lnkinf : (kind == 1) ? -T * tp[4] : (kind == 2) ? -T * tp[5] : -tp[6] * invT;
    w.tro[kTroeSlots * tr + kind] = exp_tab(arg, t.exp2t);
  }
  __syncwarp();
  // falloff, phase 2: [M], Pr = (k0/k_inf) [M], Fc and their log10
  for (int e = lane; e < 2 * NT; e += 32) {
    const int tr = e >> 1, kind = e & 1;
    const int r = t.trx[tr];
    double* q = w.tro + kTroeSlots * tr;
    double x;
    if (kind == 1) {
      const int row = t.rrow[r] & 0xffff;
      double M = Ctot;
      for (int j = t.eptr[row]; j < t.eptr[row + 1]; ++j) M = fma(t.eval[j], w.C[t.eidx[j]], M);
      x = fmax(q[0] * M, 1e-300);
      q[4] = M;
      q[5] = x;
    } else {
      const double* tp = t.troe + 8 * tr;
      x = fma(1.0 - tp[3], q[1], fma(tp[3], q[2], q[3]));
      q[6] = x;
    }
    q[7 + kind] = log_tab(x, t.logt) * (1.0 / kLn10);   // q[7] = log10 Fc, q[8] = log10 Pr
  }
  __syncwarp();
  // falloff, phase 3: ln F of the broadening factor (slot 6; the reaction pass adds it
  // to the exponent of k_inf), the factor Pr/(1+Pr) (slot 9), and with the Jacobian
  // their derivatives.  Without the Jacobian and with fewer than 32 falloff reactions,
  // lane NT (idle in this pass) inverts the mixture heat capacity in the same division
  // instruction.
  double invcpm;
  if (!JAC && NT < 32) {
    double den_in = cpm, d2 = 0.0, s2 = 0.0, P1 = 0.0, logFc = 0.0, Pr = 0.0;
    double* q = w.tro + kTroeSlots * (lane < NT ? lane : 0);
    if (lane < NT) {
      logFc = q[7];
      Pr = q[5];
      const double c = fma(-0.67, logFc, -0.4);
      const double nn = fma(-1.27, logFc, 0.75);
      const double u = q[8] + c;
      const double den = fma(-0.14, u, nn);
      d2 = den * den;
      s2 = fma(u, u, d2);
      P1 = 1.0 + Pr;
      den_in = s2 * P1;
    }
    const double inv = 1.0 / den_in;
    if (lane < NT) {
      // log F = log Fc den^2 / (den^2 + u^2) and the factor Pr/(1+Pr) share the division
      const double logF = (logFc * d2) * (P1 * inv);
      q[9] = (Pr * s2) * inv;
      q[6] = logF * kLn10;
    }
    invcpm = __shfl_sync(0xffffffffu, inv, NT);
  } else {
    invcpm = 1.0 / cpm;
  }
  for (int tr = lane; tr < NT && (JAC || NT >= 32); tr += 32) {
    double* q = w.tro + kTroeSlots * tr;
    const double logFc = q[7], Pr = q[5];
    const double c = fma(-0.67, logFc, -0.4);
    const double nn = fma(-1.27, logFc, 0.75);
    const double u = q[8] + c;
    const double den = fma(-0.14, u, nn);
    if (!JAC) {
      // log F = log Fc den^2 / (den^2 + u^2) and the factor Pr/(1+Pr), with one
      // division for both quotients
      const double d2 = den * den, s2 = fma(u, u, d2), P1 = 1.0 + Pr;
      const double inv = 1.0 / (s2 * P1);
      const double logF = (logFc * d2) * (P1 * inv);
      q[9] = (Pr * s2) * inv;
      q[6] = logF * kLn10;
    } else {
      const double invden = 1.0 / den;
      const double f1 = u * invden;
      const double g1 = fma(f1, f1, 1.0);
      const double invg = 1.0 / g1;
      const double logF = logFc * invg;
      const double invPr1 = 1.0 / (1.0 + Pr);
      q[9] = Pr * invPr1;
      const int r = t.trx[tr];
      const double* tp = t.troe + 8 * tr;
      const double dlnkinf_dT = fma(t.Ta[r], invT, t.b[r]) * invT;
      const double dlnk0_dT = fma(tp[2], invT, tp[1]) * invT;
      const double dlnPr_dT = dlnk0_dT - dlnkinf_dT;
      const double dFc_dT = -(1.0 - tp[3]) * tp[4] * q[1] - tp[3] * tp[5] * q[2] + tp[6] * invT * invT * q[3];
      const double df1_du = nn * invden * invden;
      const double df1_dnn = -u * invden * invden;
      const double dlogF_df1 = -logFc * 2.0 * f1 * invg * invg;
      const double dlogF_dx = dlogF_df1 * df1_du;
      const double dlogF_dlogFc = invg + dlogF_df1 * (df1_du * -0.67 + df1_dnn * -1.27);
      // d ln F / dT = ln10 (dlogF/dx dx/dT + dlogF/dlogFc dlogFc/dT), x = log10 Pr
      const double dlnF_dT = fma(dlogF_dx, dlnPr_dT, dlogF_dlogFc * dFc_dT / q[6]);
      q[10] = dlnPr_dT * invPr1 + dlnF_dT;            // added to d ln k_inf / dT
      q[11] = (invPr1 + dlogF_dx) / q[4];             // d ln k_f / d[M]
      q[6] = logF * kLn10;                            // (Fc, read above, is no longer needed)
    }
  }
  __syncwarp();
  // two reactions per lane per iteration: independent exponentials interleave.  The
  // table groups falloff, then third-body, then plain reactions; with at most 32 of
  // the first two kinds all of them are first reactions of the first iteration
  // (r0 < 32, the same for the whole warp), so every other slot takes the plain code.
  const bool peel = t.n_tb <= 32;
  for (int r0 = lane; r0 < R; r0 += 64) {
    const int r1 = (r0 + 32 < R) ? r0 + 32 : r0;
    RxnOut o0, o1;
    if (peel && r0 >= 32) rxn_eval<JAC, true>(t, w, r0, lnT, invT, Ctot, o0);
    else rxn_eval<JAC>(t, w, r0, lnT, invT, Ctot, o0);
    if (peel && r1 >= 32) rxn_eval<JAC, true>(t, w, r1, lnT, invT, Ctot, o1);
    else rxn_eval<JAC>(t, w, r1, lnT, invT, Ctot, o1);
    w.q[r0] = o0.q;
    if (JAC) { w.kfw[r0] = o0.kfw; w.krw[r0] = o0.krw; w.dqdT[r0] = o0.dqdT; w.tbs[r0] = o0.tbs; }
    if (r1 != r0) {
      w.q[r1] = o1.q;
      if (JAC) { w.kfw[r1] = o1.kfw; w.krw[r1] = o1.krw; w.dqdT[r1] = o1.dqdT; w.tbs[r1] = o1.tbs; }
    }
  }
  __syncwarp();
  gather_species(t, w, w.q, w.wd, lane);
  if (JAC) {
    gather_species(t, w, w.dqdT, w.DT, lane);
    gather_species(t, w, w.tbs, w.tbk, lane);
  }
  double qp = 0.0;
  for (int k = lane; k < Ns; k += 32) qp = fma(w.hh[k], w.wd[k], qp);
  s.T = T; s.invT = invT; s.lnT = lnT; s.S = S; s.invS = invS; s.rho = rho; s.invrho = invrho; s.Ctot = Ctot;
  s.Q = warp_sum(qp);
  s.cpm = cpm;
  s.invcpm = invcpm;
  __syncwarp();
}

// f^F into f[0..n): f_k = wdot_k W_k / rho, f_T = -T Q / (rho cpm).
__device__ __forceinline__ void chem_rhs_out(const Tab& t, const WS& w, const Scal& s, double* f, int lane) {
  const int Ns = t.Ns;
  for (int k = lane; k < Ns; k += 32) f[k] = w.wd[k] * t.W[k] * s.invrho;
  if (lane == 0) f[Ns] = -(s.T * s.Q) * (s.invrho * s.invcpm);
  __syncwarp();
}

// Inputs of the Jacobian assembly in the arithmetic type MT: FP64 views of the
// chem_eval<true> arrays, or FP32 copies of them for the mixed-precision form.
template <typename MT>
struct JacIn {
  const MT *C, *hh, *cp, *wd, *DT, *tbk, *kfw, *krw, *tbs, *nu, *tcv, *W, *invW, *dcp;
  MT *DC, *aux;
};

__device__ __forceinline__ JacIn<double> jac_in64(const Tab& t, const WS& w) {
  return JacIn<double>{w.C, w.hh, w.cp, w.wd, w.DT, w.tbk, w.kfw, w.krw, w.tbs, t.nu, t.tcv, t.W, t.invW, t.dcp, w.DC,
                      w.aux};
}

// FP32 copies of the per-cell Jacobian inputs (mixed-precision form).
__device__ __forceinline__ JacIn<float> jac_in32(const Tab& t, const WS& w, int lane) {
  for (int k = lane; k < t.nsv; k += 32) {
    w.C32[k] = (float)w.C[k]; w.hh32[k] = (float)w.hh[k]; w.cp32[k] = (float)w.cp[k];
    w.wd32[k] = (float)w.wd[k]; w.DT32[k] = (float)w.DT[k]; w.tbk32[k] = (float)w.tbk[k];
  }
  for (int r = lane; r < t.R; r += 32) {
    w.kfw32[r] = (float)w.kfw[r]; w.krw32[r] = (float)w.krw[r]; w.tbs32[r] = (float)w.tbs[r];
  }
  __syncwarp();
  return JacIn<float>{w.C32, w.hh32, w.cp32, w.wd32, w.DT32, w.tbk32, w.kfw32, w.krw32, w.tbs32, t.nu32, t.tcv32,
                      t.W32, t.invW32, t.dcp32, w.DC32, w.aux32};
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// Analytic Jacobian into the n x n matrix J (leading dimension ld) after
// chem_eval<true> at the same state Z.  Columns of D = nu dq/dC are owned by lanes
// (no write conflicts); then the chain rule through C(Y, T) and rho(Y, T).
template <typename MT>
__device__ __forceinline__ void chem_jac(const Tab& t, const WS& w, const double* Z, const Scal& s, MT* J,
                                         const JacIn<MT>& in, int lane) {
  const int Ns = t.Ns, ld = w.ld, nsv = t.nsv;
  for (int l = lane; l < Ns; l += 32) {
    // third-body part common to every column: sum_r nu_kr (k_f prod - k_r prod)-scale
    for (int k = 0; k < Ns; ++k) J[k * ld + l] = in.tbk[k];
    for (int e = t.cptr[l]; e < t.cptr[l + 1]; ++e) {
      const uint64_t ce = t.cent[e];
      const int r = ce & 0xffff;
      const int mf = (ce >> 16) & 0xf, mr = (ce >> 20) & 0xf;
      const int o1 = (ce >> 24) & 0xff, o2 = (ce >> 32) & 0xff, o3 = (ce >> 40) & 0xff, o4 = (ce >> 48) & 0xff;
      const MT dq = fma_t(in.kfw[r] * in.nu[mf], in.C[o1] * in.C[o2], -in.krw[r] * in.nu[mr] * (in.C[o3] * in.C[o4]));
      const uint64_t s0 = t.rsp[2 * r], s1 = t.rsp[2 * r + 1];
      const int cnt = (int)((s0 >> 48) & 0xff);
      for (int j = 0; j < cnt; ++j) {
        const int k = (s0 >> (8 * j)) & 0xff;
        const int nuv = (int)(int8_t)((s1 >> (8 * j)) & 0xff);
        J[k * ld + l] = fma_t(in.nu[nuv], dq, J[k * ld + l]);
      }
    }
    // third-body efficiencies that differ from 1
    for (int e = t.tcptr[l]; e < t.tcptr[l + 1]; ++e) {
      const int r = t.tcr[e];
      const MT sc = in.tcv[e] * in.tbs[r];
      const uint64_t s0 = t.rsp[2 * r], s1 = t.rsp[2 * r + 1];
      const int cnt = (int)((s0 >> 48) & 0xff);
      for (int j = 0; j < cnt; ++j) {
        const int k = (s0 >> (8 * j)) & 0xff;
        const int nuv = (int)(int8_t)((s1 >> (8 * j)) & 0xff);
        J[k * ld + l] = fma_t(in.nu[nuv], sc, J[k * ld + l]);
      }
    }
  }
  __syncwarp();
  // DC_k = sum_l D_kl C_l ; aux_j = sum_k h/RT_k D_kj  (sums in FP64 either way)
  double hq = 0.0, dqt = 0.0, dcpm = 0.0;
  const double T = s.T, invT = s.invT;
  for (int k = lane; k < Ns; k += 32) {
    MT acc = MT(0), col = MT(0);
    for (int l = 0; l < Ns; ++l) {
      acc = fma_t(J[k * ld + l], in.C[l], acc);
      col = fma_t(in.hh[l], J[l * ld + k], col);
    }
    in.DC[k] = acc;
    in.aux[k] = col;
    hq = fma(w.hh[k], (double)acc, hq);
    dqt += fma((w.cp[k] - w.hh[k]) * invT, w.wd[k], w.hh[k] * fma(-(double)acc, invT, w.DT[k]));
    const double dcp = fma(fma(fma(t.dcp[3 * nsv + k], T, t.dcp[2 * nsv + k]), T, t.dcp[nsv + k]), T, t.dcp[k]);
    dcpm = fma(Z[k] * t.invW[k], dcp, dcpm);
  }
  const double HQ = warp_sum(hq);
  const double dQT = warp_sum(dqt);
  const double dCPM = warp_sum(dcpm);
  __syncwarp();
  const double invS = s.invS;
  const MT inv_rhoS = (MT)(s.invrho * invS);
  const double Phi = T * s.invrho;
  const double invcpm = s.invcpm;
  const double PQc = Phi * s.Q * invcpm;
  // species rows: J_kj = (W_k / W_j)(D_kj - (DC_k - wdot_k)/(rho S)), J_kT = (W_k/rho)(DT_k - (DC_k - wdot_k)/T)
  for (int e = lane; e < Ns * Ns; e += 32) {
    const int k = e / Ns, j = e - k * Ns;
    const MT a = (in.DC[k] - in.wd[k]) * inv_rhoS;
    J[k * ld + j] = in.W[k] * in.invW[j] * (J[k * ld + j] - a);
  }
  for (int k = lane; k < Ns; k += 32)
    J[k * ld + Ns] = (MT)(t.W[k] * s.invrho * fma(-((double)in.DC[k] - w.wd[k]), invT, w.DT[k]));
  // temperature row
  for (int j = lane; j < Ns; j += 32) {
    const double dQ = s.rho * t.invW[j] * (double)in.aux[j] - invS * t.invW[j] * HQ;
    const double dPhi = Phi * invS * t.invW[j];
    J[Ns * ld + j] = (MT)(-(dPhi * s.Q * invcpm + Phi * dQ * invcpm - PQc * w.cp[j] * t.invW[j] * invcpm));
  }
  if (lane == 0) J[Ns * ld + Ns] = (MT)(-(2.0 * PQc * invT + Phi * dQT * invcpm - PQc * dCPM * invcpm));
  __syncwarp();
}

// M = I - hg J in place.
template <typename MT>
__device__ __forceinline__ void form_newton_matrix(MT* M, int n, int ld, double hg, int lane) {
  const MT h = (MT)hg;
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e - i * n;
    M[i * ld + j] = ((i == j) ? MT(1) : MT(0)) - h * M[i * ld + j];
  }
  __syncwarp();
}

// ------------------------------------------------------------------ dense LU

// Magnitudes as IEEE bit patterns: compared as integers they order non-negative
// values exactly.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long abs_bits(float v) {
  return (unsigned long long)((unsigned)__float_as_int(v) & 0x7fffffffu);
}
__device__ __forceinline__ unsigned long long inf_bits(double) { return 0x7ff0000000000000ull; }
__device__ __forceinline__ unsigned long long inf_bits(float) { return 0x7f800000ull; }

// In-place LU with partial pivoting (largest |a|; ties to the lowest row) of the
// n x n matrix A (row stride ld, n <= 128), one warp.  piv[k] is the row interchanged
// with row k at step k, dinv[k] = 1/U_kk.  Returns 0, or k + 1 when the pivot column
// k is zero or not finite (the factorisation stops there).
// The trailing update runs over the flattened (row, column) pairs of the trailing
// block, each lane stepping through its pairs without integer division.
template <bool SCALED, typename MT>
__device__ __forceinline__ int lu_factor_warp(MT* A, int n, int ld, int* piv, MT* dinv, int lane) {
  for (int k = 0; k < n; ++k) {
    // largest |a| (the IEEE bit patterns compared as integers), ties to the lowest
    // row: each lane's best, then three warp maxima (high word, low word among the
    // lanes holding the high maximum, and 127 - row among the lanes holding both)
    unsigned long long v = 0ull;
    int bi = 127;
    for (int i = k + lane; i < n; i += 32) {
      const unsigned long long a = abs_bits(A[i * ld + k]);
      if (a > v) { v = a; bi = i; }
    }
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned hmax = __reduce_max_sync(0xffffffffu, hi);
    const unsigned lmax = __reduce_max_sync(0xffffffffu, hi == hmax ? lo : 0u);
    const unsigned long long best = ((unsigned long long)hmax << 32) | lmax;
    if (best == 0ull || best >= inf_bits(MT(0))) return k + 1;
    bi = 127 - (int)__reduce_max_sync(0xffffffffu, (v == best) ? (unsigned)(127 - bi) : 0u);
    if (lane == 0) piv[k] = bi;
    if (bi != k)
      for (int j = lane; j < n; j += 32) {
        const MT a = A[k * ld + j];
        A[k * ld + j] = A[bi * ld + j];
        A[bi * ld + j] = a;
      }
    __syncwarp();
    const MT inv = MT(1) / A[k * ld + k];
    if (lane == 0) dinv[k] = inv;
    for (int i = k + 1 + lane; i < n; i += 32) A[i * ld + k] *= inv;
    __syncwarp();
    const int m = n - k - 1;
    if (m > 0) {
      int q = lane / m, r = lane - q * m;      // pair e = q m + r of the trailing block
      for (; q < m;) {
        const int i = k + 1 + q, j = k + 1 + r;
        A[i * ld + j] = fma_t(-A[i * ld + k], A[k * ld + j], A[i * ld + j]);
        r += 32;
        while (r >= m) { r -= m; ++q; }
      }
    }
    __syncwarp();
  }
  // SCALED: the strict upper triangle is scaled row by row with 1/U_kk, so the back
  // substitution of every later solve needs no multiplication by the diagonal inverse.
  if (SCALED) {
    int i = lane / n, j = lane - i * n;
    for (; i < n;) {
      if (j > i) A[i * ld + j] *= dinv[i];
      j += 32;
      while (j >= n) { j -= n; ++i; }
    }
    __syncwarp();
  }
  return 0;
}

// Solve with the factors of lu_factor_warp<SCALED>; b is overwritten by x.  SCALED
// factors hold D^-1 U above the diagonal, unscaled ones U (diagonal inverse in dinv).
template <bool SCALED, typename MT>
__device__ __forceinline__ void lu_solve_warp(const MT* A, int n, int ld, const int* piv, const MT* dinv, MT* b,
                                              int lane) {
  if (lane == 0)
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) { const MT t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncwarp();
  for (int j = 0; j < n - 1; ++j) {
    const MT xj = b[j];
    for (int i = j + 1 + lane; i < n; i += 32) b[i] = fma_t(-A[i * ld + j], xj, b[i]);
    __syncwarp();
  }
  if (SCALED) {
    for (int i = lane; i < n; i += 32) b[i] *= dinv[i];
    __syncwarp();
    for (int j = n - 1; j > 0; --j) {
      const MT xj = b[j];
      for (int i = lane; i < j; i += 32) b[i] = fma_t(-A[i * ld + j], xj, b[i]);
      __syncwarp();
    }
  } else {
    for (int j = n - 1; j >= 0; --j) {
      const MT xj = b[j] * dinv[j];
      __syncwarp();
      if (lane == 0) b[j] = xj;
      for (int i = lane; i < j; i += 32) b[i] = fma_t(-A[i * ld + j], xj, b[i]);
      __syncwarp();
    }
  }
}

// The row interchanges piv of lu_factor_warp as one permutation, in place:
// (P b)[i] = b[perm[i]].  Each lane traces its own rows back through the
// interchanges (the last one first), so no lane waits on another.
__device__ __forceinline__ void piv_to_perm(int* piv, int n, int lane) {
  int src[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int idx = lane + 32 * r;
    if (idx < n)
      for (int k = n - 1; k >= 0; --k) {
        const int pk = piv[k];
        idx = (idx == k) ? pk : ((idx == pk) ? k : idx);
      }
    src[r] = idx;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (lane + 32 * r < n) piv[lane + 32 * r] = src[r];
  __syncwarp();
}

// Solve with SCALED factors and the permutation of piv_to_perm, with the solution
// held in registers (row lane + 32 r in x[r], R = ceil(n / 32)): each step of the
// substitutions broadcasts one solved entry by a shuffle, so the chain from one step
// to the next is one FMA and one shuffle, with no shared-memory round trip.  The
// arithmetic (its order included) is that of lu_solve_warp<true>.
template <int R, typename MT>
__device__ __forceinline__ void lu_solve_regs(const MT* A, int n, int ld, const int* perm, const MT* dinv, MT* b,
                                              int lane) {
  MT x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    x[r] = (i < n) ? b[perm[i]] : MT(0);
  }
  // L y = P b (unit lower triangle)
#pragma unroll
  for (int jb = 0; jb < R; ++jb) {
    const int j1 = min(n - 1, 32 * (jb + 1));
#pragma unroll 1
    for (int j = 32 * jb; j < j1; ++j) {
      const MT xj = __shfl_sync(0xffffffffu, x[jb], j - 32 * jb);
#pragma unroll
      for (int r = jb; r < R; ++r) {
        const int i = lane + 32 * r;
        if (i > j && i < n) x[r] = fma_t(-A[i * ld + j], xj, x[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i < n) x[r] *= dinv[i];
  }
  // (D^-1 U) x = D^-1 y (unit upper triangle)
#pragma unroll
  for (int jb = R - 1; jb >= 0; --jb) {
    const int j0 = max(1, 32 * jb);
#pragma unroll 1
    for (int j = min(n - 1, 32 * jb + 31); j >= j0; --j) {
      const MT xj = __shfl_sync(0xffffffffu, x[jb], j - 32 * jb);
#pragma unroll
      for (int r = 0; r <= jb; ++r) {
        const int i = lane + 32 * r;
        if (i < j) x[r] = fma_t(-A[i * ld + j], xj, x[r]);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i < n) b[i] = x[r];
  }
  __syncwarp();
}

// 32 < n <= 64, FP64 factors: the register solve with a forward layout of its own.  With rows
// lane and 32 + lane per lane, the short block (rows 32..n-1) stays active through
// every forward step, so each step costs two FMA instructions.  The forward pass
// instead holds rows nb + lane (nb = n - 32, the long block) and rows lane < nb
// (the short block, needed only for the first nb columns): nb + (n - 1) instead of
// 32 + (n - 1) FMA instructions.  One pair of shuffles then moves the solution to
// the backward layout (rows lane and 32 + lane), where the short block is needed
// only for the last columns.  Every row receives its updates in the same order as
// in lu_solve_regs, so the results are the same.
template <typename MT>
__device__ __forceinline__ void lu_solve_regs2(const MT* A, int n, int ld, const int* perm, const MT* dinv, MT* b,
                                               int lane) {
  const int nb = n - 32;                 // 1..32
  const int ra = nb + lane;              // long-block row of this lane
  MT xa = b[perm[ra]];
  MT xb = (lane < nb) ? b[perm[lane]] : MT(0);
  // L y = P b
#pragma unroll 1
  for (int j = 0; j < nb; ++j) {         // columns held by the short block
    const MT xj = __shfl_sync(0xffffffffu, xb, j);
    if (lane > j && lane < nb) xb = fma_t(-A[lane * ld + j], xj, xb);
    xa = fma_t(-A[ra * ld + j], xj, xa);
  }
#pragma unroll 1
  for (int j = nb; j < n - 1; ++j) {     // columns held by the long block
    const MT xj = __shfl_sync(0xffffffffu, xa, j - nb);
    if (ra > j) xa = fma_t(-A[ra * ld + j], xj, xa);
  }
  xa *= dinv[ra];
  if (lane < nb) xb *= dinv[lane];
  // to rows lane (x0) and 32 + lane (x1)
  const MT ta = __shfl_sync(0xffffffffu, xa, (lane - nb) & 31);
  const MT tb = __shfl_sync(0xffffffffu, xa, (lane + 32 - nb) & 31);
  MT x0 = (lane < nb) ? xb : ta;
  MT x1 = (lane < nb) ? tb : MT(0);
  // (D^-1 U) x = D^-1 y
#pragma unroll 1
  for (int j = n - 1; j >= 32; --j) {
    const MT xj = __shfl_sync(0xffffffffu, x1, j - 32);
    x0 = fma_t(-A[lane * ld + j], xj, x0);
    if (32 + lane < j) x1 = fma_t(-A[(32 + lane) * ld + j], xj, x1);
  }
#pragma unroll 1
  for (int j = 31; j >= 1; --j) {
    const MT xj = __shfl_sync(0xffffffffu, x0, j);
    if (lane < j) x0 = fma_t(-A[lane * ld + j], xj, x0);
  }
  __syncwarp();
  b[lane] = x0;
  if (lane < nb) b[32 + lane] = x1;
  __syncwarp();
}

// The triangular solves with the permutation of piv_to_perm, in the layout `variant`
// selects (MRI_LU_*; the arithmetic and its order are the same in every layout, so
// the results are too).  Automatic: n <= 64 the register solves (FP64 factors with
// 32 < n the split forward layout, which saves FP64 instructions; FP32 factors the
// plain one, 1% faster there), larger systems the shared-memory substitutions of
// lu_solve_warp<true> after gathering P b in place.
template <typename MT>
__device__ __forceinline__ void lu_solve_perm(const MT* A, int n, int ld, const int* perm, const MT* dinv, MT* b,
                                              int lane, int variant = MRI_LU_AUTO) {
  if (variant == MRI_LU_AUTO) variant = (n > 64) ? MRI_LU_SHARED
                                        : (n > 32 && sizeof(MT) == 8) ? MRI_LU_REGS_SPLIT : MRI_LU_REGS;
  if (variant != MRI_LU_SHARED && n <= 32) {
    lu_solve_regs<1, MT>(A, n, ld, perm, dinv, b, lane);
  } else if (variant == MRI_LU_REGS && n <= 64) {
    lu_solve_regs<2, MT>(A, n, ld, perm, dinv, b, lane);
  } else if (variant == MRI_LU_REGS_SPLIT && n <= 64) {
    lu_solve_regs2<MT>(A, n, ld, perm, dinv, b, lane);
  } else {
    MT g[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) g[r] = (lane + 32 * r < n) ? b[perm[lane + 32 * r]] : MT(0);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (lane + 32 * r < n) b[lane + 32 * r] = g[r];
    __syncwarp();
    for (int j = 0; j < n - 1; ++j) {
      const MT xj = b[j];
      for (int i = j + 1 + lane; i < n; i += 32) b[i] = fma_t(-A[i * ld + j], xj, b[i]);
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) b[i] *= dinv[i];
    __syncwarp();
    for (int j = n - 1; j > 0; --j) {
      const MT xj = b[j];
      for (int i = lane; i < j; i += 32) b[i] = fma_t(-A[i * ld + j], xj, b[i]);
      __syncwarp();
    }
  }
}

// In-place Gauss-Jordan inversion with partial pivoting of the n x n matrix A (row
// stride ld, n <= 128), one warp, with the pivot rule of lu_factor_warp (largest |a| in
// the pivot column, ties to the lowest row; piv[k] the row interchanged with row k at
// step k).  On return A holds W^T, W = (P A)^-1 with P those interchanges, so that
// A^-1 b = W (P b) (piv_to_perm turns piv into P).  col: n scratch values.  Returns 0,
// or k + 1 when pivot column k is zero or not finite (the inversion stops there).
// Step k scales the pivot row by 1/a_kk (its own column taking 1/a_kk) and subtracts
// a_ik times it from every other row i, whose column k starts from 0; those (row,
// column) pairs run flattened over the lanes.  The transposition at the end lets the
// solve read a column of W^T per lane group without bank conflicts.
template <typename MT>
__device__ __forceinline__ int gj_invert_warp(MT* A, int n, int ld, int* piv, MT* col, int lane) {
  for (int k = 0; k < n; ++k) {
    unsigned long long v = 0ull;
    int bi = 127;
    for (int i = k + lane; i < n; i += 32) {
      const unsigned long long a = abs_bits(A[i * ld + k]);
      if (a > v) { v = a; bi = i; }
    }
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned hmax = __reduce_max_sync(0xffffffffu, hi);
    const unsigned lmax = __reduce_max_sync(0xffffffffu, hi == hmax ? lo : 0u);
    const unsigned long long best = ((unsigned long long)hmax << 32) | lmax;
    if (best == 0ull || best >= inf_bits(MT(0))) return k + 1;
    bi = 127 - (int)__reduce_max_sync(0xffffffffu, (v == best) ? (unsigned)(127 - bi) : 0u);
    if (lane == 0) piv[k] = bi;
    if (bi != k)
      for (int j = lane; j < n; j += 32) {
        const MT a = A[k * ld + j];
        A[k * ld + j] = A[bi * ld + j];
        A[bi * ld + j] = a;
      }
    __syncwarp();
    const MT inv = MT(1) / A[k * ld + k];
    for (int i = lane; i < n; i += 32) col[i] = A[i * ld + k];
    __syncwarp();
    for (int j = lane; j < n; j += 32) A[k * ld + j] = (j == k) ? inv : A[k * ld + j] * inv;
    __syncwarp();
    const int m = n - 1;                       // the rows other than k
    if (m > 0) {
      int q = lane / n, r = lane - q * n;      // pair e = q n + r: row q (+1 past k), column r
      for (; q < m;) {
        const int i = q + (q >= k ? 1 : 0);
        const MT base = (r == k) ? MT(0) : A[i * ld + r];
        A[i * ld + r] = fma_t(-col[i], A[k * ld + r], base);
        r += 32;
        while (r >= n) { r -= n; ++q; }
      }
    }
    __syncwarp();
  }
  // W -> W^T: the pairs (i, j), i < j, of the strict upper triangle, flattened
  {
    int i = 0, j = 1 + lane;                   // row i holds the pairs j = i + 1 .. n - 1
    while (i < n - 1 && j >= n) { const int over = j - n; ++i; j = i + 1 + over; }
    for (; i < n - 1;) {
      const MT a = A[i * ld + j];
      A[i * ld + j] = A[j * ld + i];
      A[j * ld + i] = a;
      j += 32;
      while (i < n - 1 && j >= n) { const int over = j - n; ++i; j = i + 1 + over; }
    }
  }
  __syncwarp();
  return 0;
}

// Column ranges ("chunks") into which inv_apply_warp splits each of the rem = n mod 32
// rows of its last, partial row group: the count c <= 32 / rem that minimises the
// chunk length ceil(n / c) plus the c - 1 additions of the partial sums.
__host__ __device__ inline int inv_chunk_count(int n) {
  const int rem = n % 32;
  if (rem == 0) return 1;
  int best_c = 1, best = n;
  for (int c = 2; c * rem <= 32; ++c) {
    const int cost = (n + c - 1) / c + c - 1;
    if (cost < best) { best = cost; best_c = c; }
  }
  return best_c;
}

// x = W (P b) with W^T in A (gj_invert_warp) and the permutation perm of piv_to_perm;
// b is overwritten by x.  Row 32 g + lane of a full group of 32 rows is one lane's dot
// product (two accumulators, even and odd columns); each of the rem rows of a last
// partial group is split into `chunks` column ranges on consecutive lanes, whose
// partial sums are added in chunk order.  No step waits on another lane's result
// except that final addition.
template <typename MT>
__device__ __forceinline__ void inv_apply_warp(const MT* A, int n, int ld, const int* perm, MT* b, int chunks,
                                               int lane) {
  MT g[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) g[r] = (lane + 32 * r < n) ? b[perm[lane + 32 * r]] : MT(0);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (lane + 32 * r < n) b[lane + 32 * r] = g[r];
  __syncwarp();
  const int full = n >> 5, rem = n & 31;
  MT x[4];
#pragma unroll
  for (int gi = 0; gi < 4; ++gi) {
    x[gi] = MT(0);
    if (gi < full) {
      const int i = 32 * gi + lane;
      MT a0 = MT(0), a1 = MT(0);
      int j = 0;
      for (; j + 1 < n; j += 2) {
        a0 = fma_t(A[j * ld + i], b[j], a0);
        a1 = fma_t(A[(j + 1) * ld + i], b[j + 1], a1);
      }
      if (j < n) a0 = fma_t(A[j * ld + i], b[j], a0);
      x[gi] = a0 + a1;
    }
  }
  const int c = chunks, rr = lane / c, h = lane - rr * c;
  MT sum = MT(0);
  if (rem > 0) {
    const int len = (n + c - 1) / c;
    MT acc = MT(0);
    if (rr < rem) {
      const int i = 32 * full + rr;
      const int j1 = min(n, (h + 1) * len);
      for (int j = h * len; j < j1; ++j) acc = fma_t(A[j * ld + i], b[j], acc);
    }
    sum = acc;
    for (int o = 1; o < c; ++o) {
      const MT v = __shfl_down_sync(0xffffffffu, acc, o);
      if (h + o < c) sum += v;
    }
  }
  __syncwarp();
#pragma unroll
  for (int gi = 0; gi < 4; ++gi)
    if (gi < full) b[32 * gi + lane] = x[gi];
  if (rem > 0 && h == 0 && rr < rem) b[32 * full + rr] = sum;
  __syncwarp();
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
  int ncell, K, n_sub, ramp, max_newton, nstage, sticky, jac_policy, ws_stride;
  int* queue;            // work-queue counter (zeroed before the launch)
  const double* guess;   // [ncell][n_sub][n] predicted substep ends (MRI_START_GUESS*), else null
  int start;             // MRI_START_*
  int32_t* n_fallback;   // counts Newton restarts from the previous stage value (nullable)
  const int8_t* step_exp;  // adaptive: per-cell first step exponent (nullable)
  unsigned char* mcache; // Newton-matrix cache entries (nullable), mc_stride bytes per cell
  size_t mc_stride, mc_f_off;
  int adaptive, q;       // adaptive substeps; order of the error estimate
  int schedule;          // MRI_SCHED_QUEUE or MRI_SCHED_STATIC
  int lu_variant;        // MRI_LU_*: layout of the triangular solves
  double ctrl_rtol, ctrl_atol_Y, ctrl_atol_T;
  double bhat[3];        // embedded weights of the error estimate
  unsigned long long budget_ns;   // 0: no time budget
  double Hs, hh, rtol, atol_Y, atol_T;
  float newton_safety_f;
  double A[3][3], c[3], gamma;
};

constexpr int kMaxJacAge = 12;

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
// The norm only steers the iteration (a tolerance test and contraction-rate
// estimates), so it is formed in FP32 from the FP64 vectors: 1e-7 relative on a
// number compared with 1.  Corrections beyond the FP32 range give Inf, which the
// iteration treats like an FP64 overflow.
__device__ __forceinline__ float wrms_update(const double* d, const double* Z, int n, double rtol, double atolY, double atolT,
                              int lane) {
  float acc = 0.0f;
  const float rt = (float)rtol, aY = (float)atolY, aT = (float)atolT;
  for (int k = lane; k < n; k += 32) {
    const float dk = (float)d[k];
    const float wgt = fmaf(rt, fabsf((float)Z[k] + dk), (k == n - 1) ? aT : aY);
    const float v = dk / wgt;
    acc = fmaf(v, v, acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  const float nrm = sqrtf(acc / (float)n);
  return isnan(nrm) ? INFINITY : nrm;
}

// Jacobian at Z, M = I - hg J, then its LU factors or (MRI_LU_INVERSE) the transposed
// inverse of gj_invert_warp, whose column scratch is the unused diagonal-inverse
// vector; the row interchanges are kept as a permutation (piv_to_perm).  Returns the
// factorisation's info (0 = ok).  PREC32: the assembly (from FP64 rates), the matrix
// and its factors are FP32.
template <bool PREC32>
__device__ __forceinline__ int refresh_matrix(const Tab& t, const WS& w, const double* Z, double p, double hg,
                                              int variant, int lane) {
  Scal s;
  chem_eval<true>(t, w, Z, p, s, lane);
  int rc;
  if (PREC32) {
    const JacIn<float> in = jac_in32(t, w, lane);
    chem_jac<float>(t, w, Z, s, w.M32, in, lane);
    form_newton_matrix<float>(w.M32, t.n, w.ld, hg, lane);
    rc = (variant == MRI_LU_INVERSE) ? gj_invert_warp<float>(w.M32, t.n, w.ld, w.piv, w.dinv32, lane)
                                     : lu_factor_warp<true, float>(w.M32, t.n, w.ld, w.piv, w.dinv32, lane);
  } else {
    chem_jac<double>(t, w, Z, s, w.M, jac_in64(t, w), lane);
    form_newton_matrix<double>(w.M, t.n, w.ld, hg, lane);
    rc = (variant == MRI_LU_INVERSE) ? gj_invert_warp<double>(w.M, t.n, w.ld, w.piv, w.dinv, lane)
                                     : lu_factor_warp<true, double>(w.M, t.n, w.ld, w.piv, w.dinv, lane);
  }
  if (rc == 0) piv_to_perm(w.piv, t.n, lane);
  return rc;
}

// Newton correction: d <- M^-1 d.  PREC32: the FP64 residual is rounded to FP32,
// solved with the FP32 factors and the correction widened back to FP64; the FP64
// residual of every Newton iteration then refines the stage value to the same
// tolerance as the FP64 form.
template <bool PREC32>
__device__ __forceinline__ void newton_solve(const WS& w, int n, int lane, int variant, int chunks) {
  if (PREC32) {
    for (int k = lane; k < n; k += 32) w.d32[k] = (float)w.d[k];
    __syncwarp();
    if (variant == MRI_LU_INVERSE) inv_apply_warp<float>(w.M32, n, w.ld, w.piv, w.d32, chunks, lane);
    else lu_solve_perm<float>(w.M32, n, w.ld, w.piv, w.dinv32, w.d32, lane, variant);
    for (int k = lane; k < n; k += 32) w.d[k] = (double)w.d32[k];
    __syncwarp();
  } else {
    if (variant == MRI_LU_INVERSE) inv_apply_warp<double>(w.M, n, w.ld, w.piv, w.d, chunks, lane);
    else lu_solve_perm<double>(w.M, n, w.ld, w.piv, w.dinv, w.d, lane, variant);
  }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The warp's next cell.  Queue: lane 0 takes the next index from the launch's queue
// counter, unless the warp's time budget is spent (then ncell: no cell), and broadcasts
// it.  Static: warp gw of the grid's nw warps takes cells gw, gw + nw, gw + 2 nw, ...
// (k counts the warp's cells so far).
__device__ __forceinline__ int next_cell(const StageArgs& a, unsigned long long t_start, int gw, int nw, int& k,
                                         int lane) {
  if (a.schedule == MRI_SCHED_STATIC) {
    const long long c = (long long)gw + (long long)(k++) * nw;
    return c < a.ncell ? (int)c : a.ncell;
  }
  int c = a.ncell;
  if (lane == 0 && (a.budget_ns == 0 || globaltimer_ns() - t_start < a.budget_ns)) c = atomicAdd(a.queue, 1);
  return __shfl_sync(0xffffffffu, c, 0);
}

// Step-size factor of the adaptive controller: the largest of 4, 2, 1, 1/2 not above
// 0.9 err^(-1/q), else 1/4.  Powers of two keep every substep size and offset a dyadic
// multiple of the first substep.
__device__ __forceinline__ double ctrl_factor(double err, int q) {
  const double F[4] = {4.0, 2.0, 1.0, 0.5};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double th = 0.9 / F[k];
    double thq = th;
    for (int j = 1; j < q; ++j) thq *= th;
    if (err <= thq) return F[k];
  }
  return 0.25;
}

// The cells of one stage launch, for one warp: after the CTA has staged the
// mechanism tables at smem and the SDIRK tableau at sA / sc, the warp takes cells from
// the launch's queue and integrates each over the stage (Eq. 3 with the forcing
// polynomial r_i): n_sub SDIRK substeps (plus the start-up ramp), each stage solved by
// Newton's method with the factorised matrix I - h gamma J.
template <bool PREC32>
__device__ __forceinline__ void stage_cells(const StageArgs& a, unsigned char* smem, const double (*sA)[3],
                                            const double* sc, int warp, int lane) {
  const Tab t(smem, a.L);
  const WS w(reinterpret_cast<double*>(smem + a.L.bytes) + (size_t)warp * a.ws_stride, a.L, PREC32, a.K);
  const int n = t.n, Ns = t.Ns, S = a.nstage;
  const int total_sub = a.n_sub + (a.ramp > 0 ? a.ramp : 0);
  const int chunks = inv_chunk_count(n);   // MRI_LU_INVERSE solves
  const int layout = (a.lu_variant == MRI_LU_INVERSE) ? 1 : 0;   // what a cache entry holds
  // Persistent warps take cells from a device work queue, so that cells of uneven
  // stiffness (Newton and Jacobian counts vary severalfold across a front) balance.
  // With a time budget a warp stops taking cells once it has run that long, so the
  // cells taken are always a prefix of the range.
  const unsigned long long t_start = a.budget_ns ? globaltimer_ns() : 0ull;
  const int wpb = (int)(blockDim.x >> 5);
  const int gw = (int)blockIdx.x * wpb + warp, nw = (int)gridDim.x * wpb;   // static schedule only
  int taken = 0;
  int cell = next_cell(a, t_start, gw, nw, taken, lane);
  for (; cell < a.ncell; ) {
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
    bool f_cached = false; // the cache entry holds f^F at the cell's state
    // the cell's factorised matrix from an earlier call, when the cache holds one
    unsigned char* mce = (a.mcache && a.jac_policy == MRI_JAC_LAZY && status == MRI_CELL_OK)
                             ? a.mcache + (size_t)cell * a.mc_stride : nullptr;
    if (mce) {
      const McHeader* hd = reinterpret_cast<const McHeader*>(mce);
      if (hd->tag == kMcTag && hd->n == n && hd->prec == (PREC32 ? 1 : 0) && hd->layout == layout) {
        const int nm = n * w.ld;
        if (PREC32) {
          const float* src = reinterpret_cast<const float*>(mce + sizeof(McHeader));
          for (int e = lane; e < nm; e += 32) w.M32[e] = src[e];
          for (int e = lane; e < n; e += 32) w.dinv32[e] = src[nm + e];
          const int* ps = reinterpret_cast<const int*>(src + nm + n);
          for (int e = lane; e < n; e += 32) w.piv[e] = ps[e];
        } else {
          const double* src = reinterpret_cast<const double*>(mce + sizeof(McHeader));
          for (int e = lane; e < nm; e += 32) w.M[e] = src[e];
          for (int e = lane; e < n; e += 32) w.dinv[e] = src[nm + e];
          const int* ps = reinterpret_cast<const int*>(src + nm + n);
          for (int e = lane; e < n; e += 32) w.piv[e] = ps[e];
        }
        M_hg = hd->hg;
        M_age = hd->age;
        f_cached = (hd->has_f == 1);
      }
      __syncwarp();
    }
    bool have_Fl = false;  // w.Fl holds the last stage derivative of the previous substep
    double hk_prev = 0.0;  // size of the previous substep
    // With the predictor start, f^F at the cell's state from the end of the previous
    // call (the state this call starts from, unless the caller changed it since) plus
    // this stage's forcing at its start is the derivative at the first substep's
    // start: the first stage gets a predicted Newton start too.
    if (f_cached && a.start == MRI_START_PREDICTOR) {
      const double* fc = reinterpret_cast<const double*>(mce + a.mc_f_off);
      for (int k = lane; k < n; k += 32) w.Fl[k] = fc[k] + (a.K > 0 ? w.phi[k] : 0.0);
      __syncwarp();
      have_Fl = true;
    }
    bool step_failed = false;   // adaptive: Newton failed in the current step
    // adaptive substeps: time reached within the stage, next size, attempts so far
    double t_ad = 0.0, hc = a.hh;
    if (a.adaptive && a.step_exp) hc = ldexp(a.hh, min(10, max(-20, (int)a.step_exp[cell])));
    int attempts = 0;
    for (int sidx = 0; status == MRI_CELL_OK; ++sidx) {
      double tau, hk;
      bool last_ad = false;
      if (a.adaptive) {
        if (!(t_ad < a.Hs)) break;
        if (hc < ldexp(a.Hs, -40) || attempts >= 10000) { status = MRI_CELL_ENEWTON; break; }
        ++attempts;
        last_ad = (t_ad + hc >= a.Hs * (1.0 - 1e-12));
        hk = last_ad ? a.Hs - t_ad : hc;
        tau = t_ad;
      } else {
        if (sidx >= total_sub) break;
        substep_geometry(sidx, a.ramp, a.hh, tau, hk);
      }
      const double hg = hk * a.gamma;
      const double inv_hg = 1.0 / hg;
      const bool startup_sub = (!a.adaptive && a.ramp > 0 && sidx <= a.ramp);
      // MRI_JAC_PER_SUBSTEP: Jacobian + LU at every substep start.  MRI_JAC_LAZY: the
      // factorised matrix carries over while h gamma is unchanged and it is younger
      // than kMaxJacAge substeps; poor contraction refreshes it inside Newton.
      // "Unchanged" allows rounding: stages of equal substeps compute h from their own
      // lengths (H/3 / 4 and 5H/12 / 5 differ in the last bit), and a matrix whose h gamma
      // is off by an ulp is as good a Newton matrix as the exact one.
      const bool need = (a.jac_policy == MRI_JAC_PER_SUBSTEP) || startup_sub ||
                        !(fabs(hg - M_hg) <= 1e-12 * hg) || M_age >= kMaxJacAge;
      if (need) {
        if (refresh_matrix<PREC32>(t, w, w.y0, p, hg, a.lu_variant, lane) != 0) { status = MRI_CELL_ENEWTON; break; }
        njac++;
        M_hg = hg;
        M_age = 0;
      } else {
        M_age++;
      }
      for (int i = 0; i < S && status == MRI_CELL_OK; ++i) {
        const double rh = (tau + sc[i] * hk) / a.Hs;
        // Start of Newton (a.start):
        //  MRI_START_PREDICTOR: base + h gamma F_pred, the stage equation with the new
        //    stage derivative replaced by its linear extrapolation in time from the
        //    last two known ones (the last one alone where only one is known; the
        //    previous substep's for the first stage); the previous stage value while
        //    no derivative is known yet;
        //  MRI_START_PREVIOUS: the previous stage value (y_n for the first stage);
        //  MRI_START_GUESS: the caller's predicted stage output interpolated to the
        //    stage time, y_in + rhohat (guess - y_in);
        //  MRI_START_GUESS_FIRST: the guess where the predictor has no derivative.
        int src;   // 0 predictor, 1 previous stage value, 2 guess
        if (a.start == MRI_START_PREVIOUS) src = 1;
        else if (a.start == MRI_START_GUESS) src = 2;
        else if ((i > 0) || have_Fl) src = 0;
        else src = (a.start == MRI_START_GUESS_FIRST) ? 2 : 1;
        const bool predicted = (src != 1);
        const double* Fp = (i > 0) ? w.F(i - 1) : w.Fl;
        // second point of the extrapolation and its weight: F_pred = Fp + coef (Fp - Fq).
        // For the first stage the previous substep's second-to-last stage derivative
        // (still in F(S-2)) serves when that substep had the same size; for the second
        // stage the derivative at the substep start, Fl; then the two stages before.
        // Start-up substeps keep the last derivative alone: far from the fast manifold
        // the extrapolated start can lead Newton to another root of the stage equation.
        const double* Fq = nullptr;
        double coef = 0.0;
        if (startup_sub) {
        } else if (i == 0) {
          if (have_Fl && hk == hk_prev && S >= 2) { Fq = w.F(S - 2); coef = sc[0] / (1.0 - sc[S - 2]); }
        } else if (i == 1) {
          if (have_Fl) { Fq = w.Fl; coef = (sc[1] - sc[0]) / sc[0]; }
        } else {
          Fq = w.F(i - 2);
          coef = (sc[i] - sc[i - 1]) / (sc[i - 1] - sc[i - 2]);
        }
        for (int k = lane; k < n; k += 32) {
          double rv = 0.0;
          for (int j = a.K - 1; j >= 0; --j) rv = fma(rv, rh, w.phi[j * w.nv + k]);
          w.r[k] = rv;
          double bs = w.y0[k];
          for (int j = 0; j < i; ++j) bs = fma(hk * sA[i][j], w.F(j)[k], bs);
          w.base[k] = bs;   // stage base y_n + h sum_j a_ij F_j
          double z;
          if (src == 0) {
            const double fp = Fp[k];
            z = fma(hg, Fq ? fma(coef, fp - Fq[k], fp) : fp, bs);
          } else if (src == 1) {        // Z_{i-1} = y_n + h sum_{j<i} a_{i-1,j} F_j
            z = w.y0[k];
            for (int j = 0; j < i; ++j) z = fma(hk * sA[i - 1][j], w.F(j)[k], z);
          } else {                      // between the predicted substep ends j-1 and j
            const double th = (tau + sc[i] * hk) / a.hh;
            int j = (int)th;
            if (j > a.n_sub - 1) j = a.n_sub - 1;
            const double* gc = a.guess + (size_t)cell * a.n_sub * n;
            const double lo = (j == 0) ? yc[k] : gc[(size_t)(j - 1) * n + k];
            z = fma(th - (double)j, gc[(size_t)j * n + k] - lo, lo);
          }
          w.Z[k] = z;
        }
        __syncwarp();
        // Modified Newton: the matrix of the substep start is reused while it
        // contracts.  When an iteration contracts poorly (or leaves the finite
        // range) with a matrix older than the current iterate, the iteration is
        // redone with a fresh Jacobian at the current iterate (a full Newton step;
        // the residual is reused).  Start-up substeps use full Newton throughout.
        // The converged stage value does not depend on the matrix policy.
        // If Newton fails from the predicted start, the stage is solved once more
        // with full Newton from the previous stage value (the substep start for the
        // first stage): far from the fast manifold a large F_prev can throw the
        // predicted start out of Newton's region of convergence.
        bool startup = startup_sub;
        bool fresh = (i == 0) && need && !predicted;   // matrix evaluated at the starting iterate (y_n)
        bool conv = false;
        float prev = 0.0f;       // the iteration's control quantities are FP32, like the norm
        for (int attempt = 0; attempt < 2 && !conv; ++attempt) {
        if (attempt == 1) {
          if (!predicted) break;      // the start was already the previous stage value
          if (a.n_fallback && lane == 0) atomicAdd(a.n_fallback, 1);
          for (int k = lane; k < n; k += 32) {   // Z_{i-1} = y_n + h sum_{j<i} a_{i-1,j} F_j
            double z = w.y0[k];
            for (int j = 0; j < i; ++j) z = fma(hk * sA[i - 1][j], w.F(j)[k], z);
            w.Z[k] = z;
          }
          __syncwarp();
          startup = true;
          fresh = false;
          prev = 0.0f;
        }
        for (int it = 0; it < a.max_newton; ++it) {
          Scal s;
          chem_eval<false>(t, w, w.Z, p, s, lane);
          // residual base + hg (f^F(Z) + r) - Z, with f^F formed in place (the formulas
          // of chem_rhs_out): f_k = (wdot_k W_k) / rho, f_T = (-T Q / cpm) / rho
          const double fT_rho = -(s.T * s.Q) * s.invcpm;
          for (int k = lane; k < n; k += 32) {
            const double a = (k < Ns) ? w.wd[k] * t.W[k] : fT_rho;
            const double g = fma(hg, fma(a, s.invrho, w.r[k]), w.base[k]) - w.Z[k];
            w.res[k] = g;
            w.d[k] = g;
          }
          __syncwarp();
          if (startup && !fresh) {   // start-up substeps: full Newton, as far from the manifold
            if (refresh_matrix<PREC32>(t, w, w.Z, p, hg, a.lu_variant, lane) != 0) break;
            njac++;
            fresh = true;
          }
          newton_solve<PREC32>(w, n, lane, a.lu_variant, chunks);
          float nrm = wrms_update(w.d, w.Z, n, a.rtol, a.atol_Y, a.atol_T, lane);
          // redo with a fresh matrix when the stale one contracts by less than 10x, or
          // when its contraction rate would not reach the tolerance three iterations
          // before max_newton
          bool redo = !fresh && (!isfinite(nrm) || (it > 0 && nrm > 0.1f * prev));
          if (!fresh && !redo && it > 0 && nrm > 1.0f) {
            const float rho = nrm / prev;
            float proj = nrm;
            const int left = a.max_newton - 3 - (it + 1);
            for (int j = 0; j < left && proj > 1.0f; ++j) proj *= rho;
            redo = proj > 1.0f;
          }
          if (redo) {
            if (refresh_matrix<PREC32>(t, w, w.Z, p, hg, a.lu_variant, lane) != 0) break;
            njac++;
            M_age = 0;
            for (int k = lane; k < n; k += 32) w.d[k] = w.res[k];
            __syncwarp();
            newton_solve<PREC32>(w, n, lane, a.lu_variant, chunks);
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
          // (a correction that is exactly zero has nothing left to converge)
          // (prev > 0 here: a zero correction is accepted when it occurs)
          if (nrm == 0.0f ||
              (full_step ? (nrm <= 1.0f) : (it > 0 && nrm <= 1.0f && nrm * nrm <= a.newton_safety_f * prev))) {
            conv = true;
            break;
          }
          prev = nrm;
        }
        }
        if (!conv) {
          if (a.adaptive) step_failed = true;   // repeated at a quarter of the size
          else status = MRI_CELL_ENEWTON;
          break;
        }
        double* Fi = (i < S - 1) ? w.F(i) : w.Fl;
        for (int k = lane; k < n; k += 32) Fi[k] = (w.Z[k] - w.base[k]) * inv_hg;
        __syncwarp();
      }
      if (status != MRI_CELL_OK) break;
      if (a.adaptive) {
        // embedded estimate h sum_i (b_i - bhat_i) F_i (b_i = a_{s,i}) in the WRMS norm of
        // the controller's tolerances at the new state; FP64, as it decides the steps
        double err = 0.0;
        if (!step_failed) {
          double acc = 0.0;
          for (int k = lane; k < n; k += 32) {
            double e = 0.0;
            for (int j = 0; j < S; ++j) e = fma(sA[S - 1][j] - a.bhat[j], (j < S - 1) ? w.F(j)[k] : w.Fl[k], e);
            e *= hk;
            const double wgt = fma(a.ctrl_rtol, fabs(w.Z[k]), (k == n - 1) ? a.ctrl_atol_T : a.ctrl_atol_Y);
            const double v = e / wgt;
            acc = fma(v, v, acc);
          }
          err = sqrt(warp_sum(acc) / n);
        }
        const double fac = step_failed ? 0.25 : ctrl_factor(err, a.q);
        if (step_failed || !(err <= 1.0)) {   // rejected: the state stays at the step's start
          hc = hk * fac;
          have_Fl = false;
          step_failed = false;
          continue;
        }
        t_ad = last_ad ? a.Hs : t_ad + hk;
        hc = fmin(hk * fac, a.Hs);
      }
      for (int k = lane; k < n; k += 32) w.y0[k] = w.Z[k];
      __syncwarp();
      have_Fl = true;
      hk_prev = hk;
      nsub++;
    }
    if (mce && status == MRI_CELL_OK && M_hg != 0.0) {   // keep the matrix for the next call
      McHeader* hd = reinterpret_cast<McHeader*>(mce);
      if (njac > 0) {
        const int nm = n * w.ld;
        if (PREC32) {
          float* dst = reinterpret_cast<float*>(mce + sizeof(McHeader));
          for (int e = lane; e < nm; e += 32) dst[e] = w.M32[e];
          for (int e = lane; e < n; e += 32) dst[nm + e] = w.dinv32[e];
          int* pd = reinterpret_cast<int*>(dst + nm + n);
          for (int e = lane; e < n; e += 32) pd[e] = w.piv[e];
        } else {
          double* dst = reinterpret_cast<double*>(mce + sizeof(McHeader));
          for (int e = lane; e < nm; e += 32) dst[e] = w.M[e];
          for (int e = lane; e < n; e += 32) dst[nm + e] = w.dinv[e];
          int* pd = reinterpret_cast<int*>(dst + nm + n);
          for (int e = lane; e < n; e += 32) pd[e] = w.piv[e];
        }
      }
      // f^F at the output state: the last stage derivative less the forcing it included
      double* fc = reinterpret_cast<double*>(mce + a.mc_f_off);
      for (int k = lane; k < n; k += 32) fc[k] = w.Fl[k] - w.r[k];
      if (lane == 0) {
        hd->hg = M_hg;
        hd->age = M_age;
        hd->n = n;
        hd->prec = PREC32 ? 1 : 0;
        hd->has_f = (nsub > 0) ? 1 : 0;
        hd->layout = layout;
        hd->tag = kMcTag;
      }
    } else if (mce && lane == 0) {
      reinterpret_cast<McHeader*>(mce)->tag = 0;       // a failed cell leaves no matrix behind
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
    cell = next_cell(a, t_start, gw, nw, taken, lane);
  }
}

// The launch is planned at one CTA per SM or more, each of at most kMaxWarps warps;
// the minimum of one block lets ptxas spend the whole per-thread register budget
// (without it ptxas settles on far fewer registers and spills).
template <bool PREC32>
__global__ void __launch_bounds__(kMaxWarps * 32, 1) stage_fast_kernel(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sA[3][3], sc[3];    // SDIRK tableau, indexed by the runtime stage
  stage_table(smem, a.table, a.L.bytes);
  if (threadIdx.x < 9) sA[threadIdx.x / 3][threadIdx.x % 3] = a.A[threadIdx.x / 3][threadIdx.x % 3];
  if (threadIdx.x < 3) sc[threadIdx.x] = a.c[threadIdx.x];
  __syncthreads();
  stage_cells<PREC32>(a, smem, sA, sc, threadIdx.x >> 5, threadIdx.x & 31);
}

// Tableau of an explicit fast method (Sec. 3.2: the paper's MRI-P(k) runs use explicit
// Runge-Kutta fast methods): K_i = F(tau + c_i h, y + h sum_{j<i} a_ij K_j),
// y <- y + h sum_i b_i K_i, s <= 4 stages.
struct ErkArgs {
  double A[4][4], b[4], c[4];
  int s;
};

// The cells of one stage launch with an explicit fast method, for one warp: n_sub
// substeps (plus the start-up sequence), each with s evaluations of f^F + r(theta) and
// the weighted update; no Jacobian, no Newton iteration.  A substep whose new state is
// not finite leaves the cell at the state before it with MRI_CELL_ENEWTON.
// cell_stats[1] counts right-hand-side evaluations.
__device__ __forceinline__ void stage_cells_explicit(const StageArgs& a, const ErkArgs& e, unsigned char* smem,
                                                     int warp, int lane) {
  const Tab t(smem, a.L);
  const WS w(reinterpret_cast<double*>(smem + a.L.bytes) + (size_t)warp * a.ws_stride, a.L, false, a.K, false);
  const int n = t.n, Ns = t.Ns, S = e.s;
  const int total_sub = a.n_sub + (a.ramp > 0 ? a.ramp : 0);
  const int wpb = (int)(blockDim.x >> 5);
  const int gw = (int)blockIdx.x * wpb + warp, nw = (int)gridDim.x * wpb;
  int taken = 0;
  const unsigned long long t_start = a.budget_ns ? globaltimer_ns() : 0ull;
  int cell = next_cell(a, t_start, gw, nw, taken, lane);
  for (; cell < a.ncell; ) {
    double* yc = a.y + (size_t)cell * n;
    const double p = a.p[cell];
    int bad = 0;
    for (int k = lane; k < n; k += 32) {
      const double v = yc[k];
      w.y0[k] = v;
      if (!isfinite(v)) bad = 1;
    }
    for (int q = lane; q < a.K * n; q += 32) w.phi[(q / n) * w.nv + (q % n)] = a.phi[(size_t)cell * a.K * n + q];
    __syncwarp();
    bad = __any_sync(0xffffffffu, bad) || !(w.y0[Ns] > 0.0) || !(p > 0.0) || !isfinite(p);
    int status = bad ? MRI_CELL_EINPUT : MRI_CELL_OK;
    int nsub = 0, nrhs = 0;
    for (int sidx = 0; sidx < total_sub && status == MRI_CELL_OK; ++sidx) {
      double tau, hk;
      substep_geometry(sidx, a.ramp, a.hh, tau, hk);
      for (int i = 0; i < S; ++i) {
        const double rh = (tau + e.c[i] * hk) / a.Hs;
        for (int k = lane; k < n; k += 32) {
          double z = w.y0[k];
          for (int j = 0; j < i; ++j) {
            const double* Kj = (j == 0) ? w.F0 : (j == 1) ? w.F1 : w.Fl;
            z = fma(hk * e.A[i][j], Kj[k], z);
          }
          w.Z[k] = z;
          double rv = 0.0;
          for (int q = a.K - 1; q >= 0; --q) rv = fma(rv, rh, w.phi[q * w.nv + k]);
          w.r[k] = rv;
        }
        __syncwarp();
        Scal sc;
        chem_eval<false>(t, w, w.Z, p, sc, lane);
        chem_rhs_out(t, w, sc, w.f, lane);
        double* Ki = (i == 0) ? w.F0 : (i == 1) ? w.F1 : w.Fl;   // K_3 is only summed
        for (int k = lane; k < n; k += 32) {
          const double kv = w.f[k] + w.r[k];
          if (i < S - 1) Ki[k] = kv;
          w.res[k] = (i == 0) ? e.b[0] * kv : fma(e.b[i], kv, w.res[k]);
        }
        __syncwarp();
        ++nrhs;
      }
      int fin = 1;
      for (int k = lane; k < n; k += 32) {
        const double v = fma(hk, w.res[k], w.y0[k]);
        w.Z[k] = v;
        if (!isfinite(v)) fin = 0;
      }
      if (!__all_sync(0xffffffffu, fin)) {
        status = MRI_CELL_ENEWTON;     // the cell keeps the state before this substep
        break;
      }
      for (int k = lane; k < n; k += 32) w.y0[k] = w.Z[k];
      __syncwarp();
      ++nsub;
    }
    if (status != MRI_CELL_EINPUT)
      for (int k = lane; k < n; k += 32) yc[k] = w.y0[k];
    if (lane == 0) {
      if (a.status && (!a.sticky || status != MRI_CELL_OK)) a.status[cell] = status;
      if (a.stats) {
        int32_t* st = a.stats + 4 * (size_t)cell;
        st[0] += nsub; st[1] += nrhs; st[3] += (status != MRI_CELL_OK);
      }
      if (a.n_failed && status != MRI_CELL_OK) atomicAdd(a.n_failed, 1);
    }
    __syncwarp();
    cell = next_cell(a, t_start, gw, nw, taken, lane);
  }
}

__global__ void __launch_bounds__(kMaxWarps * 32, 1) stage_explicit_kernel(StageArgs a, ErkArgs e) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table(smem, a.table, a.L.bytes);
  __syncthreads();
  stage_cells_explicit(a, e, smem, threadIdx.x >> 5, threadIdx.x & 31);
}

// Several mechanisms in one launch: CTAs [block0[g], block0[g+1]) serve group g, each
// with its own staged tables, workspace layout and queue.  The group's arguments are
// copied to shared memory so that the hot loop reads them from there.
struct BatchArgs {
  StageArgs g[MRI_MAX_GROUPS];
  int block0[MRI_MAX_GROUPS + 1];
  int warps[MRI_MAX_GROUPS];
  int ngroups;
};
static_assert(sizeof(BatchArgs) <= 32764, "batch arguments must fit the kernel parameter space");
static_assert(sizeof(StageArgs) + 12 * sizeof(double) <= 1024, "static shared memory of the stage kernels");

template <bool PREC32>
// The split of the CTAs is only where they start: a CTA whose group has no cells left
// moves on to the other groups in turn (staging their tables), so the groups whose cells
// cost most get help at the end instead of leaving the other SMs idle.  Every cell is
// still integrated by one warp with its group's tables, so results do not change.
__global__ void __launch_bounds__(kMaxWarps * 32) stage_fast_batch_kernel(const __grid_constant__ BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sA[3][3], sc[3];
  __shared__ StageArgs sa;
  int gi = 0;
  while (gi + 1 < b.ngroups && (int)blockIdx.x >= b.block0[gi + 1]) ++gi;
  const int warp = threadIdx.x >> 5;
  for (int pass = 0; pass < b.ngroups; ++pass) {
    const int g = (gi + pass) % b.ngroups;
    if (threadIdx.x == 0) sa = b.g[g];
    stage_table(smem, b.g[g].table, b.g[g].L.bytes);
    if (threadIdx.x < 9) sA[threadIdx.x / 3][threadIdx.x % 3] = b.g[g].A[threadIdx.x / 3][threadIdx.x % 3];
    if (threadIdx.x < 3) sc[threadIdx.x] = b.g[g].c[threadIdx.x];
    __syncthreads();
    if (warp < b.warps[g]) stage_cells<PREC32>(sa, smem, sA, sc, warp, threadIdx.x & 31);
    __syncthreads();        // every warp is done with this group's tables before the next are staged
  }
}

// Cells the budget left untaken: [min(counter, ncell), ncell).
__global__ void mark_untaken_kernel(const int* queue, int ncell, int32_t* status, int32_t* n_failed) {
  const int first = min(*queue, ncell);
  for (int c = first + blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
    if (status) status[c] = MRI_CELL_TIMEOUT;
  if (n_failed && blockIdx.x == 0 && threadIdx.x == 0 && ncell > first) atomicAdd(n_failed, ncell - first);
}

// ------------------------------------------------------------------ per-kernel entry kernels

__global__ void __launch_bounds__(kMaxWarps * 32) rhs_kernel(const double* y, const double* p, int ncell,
                                                              double* f, const unsigned char* table, Layout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_table(smem, table, L.bytes);
  __syncthreads();
  const Tab t(smem, L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const WS w(reinterpret_cast<double*>(smem + L.bytes) + (size_t)warp * ws_offsets(L, false, 0).total, L, false, 0);
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
  const WS w(reinterpret_cast<double*>(smem + L.bytes) + (size_t)warp * ws_offsets(L, false, 0).total, L, false, 0);
  const int n = t.n;
  for (int cell = blockIdx.x * nw + warp; cell < ncell; cell += gridDim.x * nw) {
    for (int k = lane; k < n; k += 32) w.Z[k] = y[(size_t)cell * n + k];
    __syncwarp();
    Scal s;
    chem_eval<true>(t, w, w.Z, p[cell], s, lane);
    chem_jac<double>(t, w, w.Z, s, w.M, jac_in64(t, w), lane);
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
    const int rc = lu_factor_warp<false, double>(Ms, n, ld, pv, dv, lane);
    if (rc == 0) lu_solve_warp<false, double>(Ms, n, ld, pv, dv, bs, lane);
    for (int e = lane; e < n * n; e += 32) A[(size_t)sys * n * n + e] = Ms[(e / n) * ld + e % n];
    for (int k = lane; k < n; k += 32) b[(size_t)sys * n + k] = bs[k];
    if (lane == 0 && info) info[sys] = rc;
    __syncwarp();
  }
}

// The inverse path of MRI_LU_INVERSE on a batch of FP64 systems (one warp per system):
// A <- A^-1 (row-major, from W^T: A^-1[i][perm[k]] = W[i][k]), b <- W (P b).
__global__ void inverse_kernel(double* A, double* b, int n, int ld, int nbatch, int32_t* info) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = round_up(n * ld, 2) + 2 * round_up(n, 2) + n;
  double* Ms = reinterpret_cast<double*>(smem) + (size_t)warp * per;
  double* bs = Ms + round_up(n * ld, 2);
  double* cs = bs + round_up(n, 2);
  int* pv = reinterpret_cast<int*>(cs + round_up(n, 2));
  const int chunks = inv_chunk_count(n);
  for (int sys = blockIdx.x * nw + warp; sys < nbatch; sys += gridDim.x * nw) {
    for (int e = lane; e < n * n; e += 32) Ms[(e / n) * ld + e % n] = A[(size_t)sys * n * n + e];
    for (int k = lane; k < n; k += 32) bs[k] = b[(size_t)sys * n + k];
    __syncwarp();
    const int rc = gj_invert_warp<double>(Ms, n, ld, pv, cs, lane);
    if (rc == 0) {
      piv_to_perm(pv, n, lane);
      inv_apply_warp<double>(Ms, n, ld, pv, bs, chunks, lane);
      for (int e = lane; e < n * n; e += 32) {
        const int k = e / n, i = e % n;        // W^T[k][i] = W[i][k] -> A^-1[i][perm[k]]
        A[(size_t)sys * n * n + (size_t)i * n + pv[k]] = Ms[k * ld + i];
      }
      for (int k = lane; k < n; k += 32) b[(size_t)sys * n + k] = bs[k];
    }
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

// Raise a kernel's dynamic shared memory limit to the device's opt-in maximum, once per
// kernel and device, so that later launches (also those recorded by a stream capture)
// make no attribute call.
static bool allow_full_smem(const void* fn) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first == fn && d.second == dev) return true;
  // the opt-in limit covers static and dynamic shared memory together
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           device_smem_limit() - (int)fa.sharedSizeBytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  done.emplace_back(fn, dev);
  return true;
}

static int device_sm_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  return v > 0 ? v : 48 * 1024;
}

// Warps per CTA and grid for a warp-per-cell kernel with `per_warp` bytes of workspace
// after the staged table.  wpb / bps: requested warps per CTA and CTAs per SM (0 =
// automatic).  The grid is persistent: at most bps CTAs per SM.
// Static shared memory of the kernels, at most: the batched kernel (tableau and a
// group's arguments) and the single-mechanism stage kernels (the tableau, 96 bytes).
constexpr long long kStaticSmem = 1024;
constexpr long long kStageStaticSmem = 128;

static bool plan_launch(const Layout& L, int ncell, int& warps, int& blocks, size_t& smem, bool prec32 = false,
                        int K = 0, int wpb = 0, int bps = 0, bool matrix = true,
                        long long static_smem = kStaticSmem) {
  constexpr long long kReservedPerCta = 1024;   // shared memory the SM keeps per resident CTA
  const int per_cta_sm = bps > 0 ? bps : 1;
  long long cap = device_smem_limit();
  const long long share = (long long)device_sm_smem() / per_cta_sm - kReservedPerCta;
  if (share < cap) cap = share;
  const size_t per_warp = (size_t)ws_offsets(L, prec32, K, matrix).total * 8;
  long long room = cap - static_smem - (long long)L.bytes;
  int wmax = room > 0 ? (int)(room / (long long)per_warp) : 0;
  if (wmax > kMaxWarps) wmax = kMaxWarps;
  if (wmax < 1) return false;
  const int slots = device_sm_count() * per_cta_sm;
  if (wpb > 0) {
    if (wpb > wmax) return false;
    warps = wpb;
  } else {
    int want = (ncell + slots - 1) / slots;
    warps = want < 1 ? 1 : (want > wmax ? wmax : want);
  }
  blocks = (ncell + warps - 1) / warps;
  if (blocks > slots) blocks = slots;
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
    // first-order embedded weights (1, 0): the estimate is h gamma (F_2 - F_1)
    a.bhat[0] = 1.0; a.bhat[1] = 0.0; a.bhat[2] = 0.0;
    a.q = 2;
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
    // second-order embedded weights on the first two stages: sum 1, bhat . c = 1/2
    a.bhat[1] = (0.5 - a.c[0]) / (a.c[1] - a.c[0]);
    a.bhat[0] = 1.0 - a.bhat[1];
    a.bhat[2] = 0.0;
    a.q = 3;
  }
}

bool is_explicit(int method) { return method == MRI_ERK2 || method == MRI_ERK3 || method == MRI_ERK4; }

// Heun (order 2), Kutta's third-order method and the classical fourth-order method.
static ErkArgs erk_table(int method) {
  ErkArgs e{};
  if (method == MRI_ERK2) {
    e.s = 2;
    e.A[1][0] = 1.0;
    e.b[0] = 0.5; e.b[1] = 0.5;
    e.c[1] = 1.0;
  } else if (method == MRI_ERK3) {
    e.s = 3;
    e.A[1][0] = 0.5;
    e.A[2][0] = -1.0; e.A[2][1] = 2.0;
    e.b[0] = 1.0 / 6.0; e.b[1] = 2.0 / 3.0; e.b[2] = 1.0 / 6.0;
    e.c[1] = 0.5; e.c[2] = 1.0;
  } else {
    e.s = 4;
    e.A[1][0] = 0.5; e.A[2][1] = 0.5; e.A[3][2] = 1.0;
    e.b[0] = 1.0 / 6.0; e.b[1] = 1.0 / 3.0; e.b[2] = 1.0 / 3.0; e.b[3] = 1.0 / 6.0;
    e.c[1] = 0.5; e.c[2] = 0.5; e.c[3] = 1.0;
  }
  return e;
}

// Arguments of one stage launch over the cells of one mechanism.
static int fill_stage_args(StageArgs& a, double* y, const double* p, int ncell, const double* phi, int K,
                           double Hs, double h, const Mech& m, const mri_fast_opts& o, int ramp, int32_t* status,
                           int32_t* stats, int32_t* n_failed, bool sticky) {
  a = StageArgs{};
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
  a.newton_safety_f = (float)o.newton_safety;
  if (!is_explicit(o.method)) sdirk_table(o.method, a);
  a.ws_stride = is_explicit(o.method) ? ws_offsets(m.L, false, K, false).total
                                      : ws_offsets(m.L, o.precision == MRI_PREC_FP32_LU, K).total;
  a.budget_ns = o.time_budget_s > 0 ? (unsigned long long)std::ceil(o.time_budget_s * 1e9) : 0ull;
  a.adaptive = o.adaptive;
  a.schedule = o.schedule;
  a.lu_variant = o.lu_variant;
  a.ctrl_rtol = o.ctrl_rtol; a.ctrl_atol_Y = o.ctrl_atol_Y; a.ctrl_atol_T = o.ctrl_atol_T;
  if (o.adaptive) a.ramp = 0;   // the controller finds its own start-up steps
  if (o.matrix_cache) {
    a.mc_stride = mc_stride(m.L, o.precision == MRI_PREC_FP32_LU);
    a.mc_f_off = mc_f_offset(m.L, o.precision == MRI_PREC_FP32_LU);
    if (o.matrix_cache_bytes < a.mc_stride * (size_t)ncell) return MRI_EINVAL;
    a.mcache = static_cast<unsigned char*>(o.matrix_cache);
  }
  return MRI_OK;
}

// Each launch takes its own counter of the mechanism's ring, so that launches in
// flight on different streams do not share one (up to kQueueSlots of them); the
// counter is zeroed in stream order before the launch.  A launch recorded under stream
// capture takes a counter from the second ring, which eager launches never use: the
// graph keeps that counter for every replay, so eager launches that wrap their own
// ring cannot collide with a replay in flight.
static int take_queue(const Mech& m, StageArgs& a, cudaStream_t st) {
  Mech& mm = const_cast<Mech&>(m);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MRI_ECUDA;
  if (cap == cudaStreamCaptureStatusNone)
    a.queue = mm.d_queue + (__atomic_fetch_add(&mm.queue_next, 1u, __ATOMIC_RELAXED) % kQueueSlots);
  else
    a.queue = mm.d_queue + kQueueSlots +
              (__atomic_fetch_add(&mm.graph_next, 1u, __ATOMIC_RELAXED) % kGraphQueueSlots);
  return cudaMemsetAsync(a.queue, 0, sizeof(int), st) == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

int launch_stage_fast(double* y, const double* p, int ncell, const double* phi, int K, double Hs, double h,
                      const Mech& m, const mri_fast_opts& o, int ramp, int32_t* status, int32_t* stats,
                      int32_t* n_failed, cudaStream_t st, bool sticky, const double* guess, int start,
                      int32_t* n_fallback, const int8_t* step_exp) {
  if (ncell == 0) return MRI_OK;
  StageArgs a;
  int rc = fill_stage_args(a, y, p, ncell, phi, K, Hs, h, m, o, ramp, status, stats, n_failed, sticky);
  if (rc != MRI_OK) return rc;
  a.guess = guess;
  a.start = start;
  a.n_fallback = n_fallback;
  a.step_exp = step_exp;
  const bool prec32 = (o.precision == MRI_PREC_FP32_LU);
  const bool expl = is_explicit(o.method);
  int warps, blocks;
  size_t smem;
  if (!plan_launch(m.L, ncell, warps, blocks, smem, prec32 && !expl, K, o.warps_per_block, o.blocks_per_sm, !expl,
                   kStageStaticSmem))
    return MRI_EINVAL;
  if ((rc = take_queue(m, a, st)) != MRI_OK) return rc;
  if (expl) {
    if (!allow_full_smem((const void*)stage_explicit_kernel)) return MRI_ECUDA;
    stage_explicit_kernel<<<blocks, warps * 32, smem, st>>>(a, erk_table(o.method));
  } else if (prec32) {
    if (!allow_full_smem((const void*)stage_fast_kernel<true>)) return MRI_ECUDA;
    stage_fast_kernel<true><<<blocks, warps * 32, smem, st>>>(a);
  } else {
    if (!allow_full_smem((const void*)stage_fast_kernel<false>)) return MRI_ECUDA;
    stage_fast_kernel<false><<<blocks, warps * 32, smem, st>>>(a);
  }
  if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  if (a.budget_ns) {
    const int nb = (ncell + 255) / 256 < 1024 ? (ncell + 255) / 256 : 1024;
    mark_untaken_kernel<<<nb, 256, 0, st>>>(a.queue, ncell, status, n_failed);
    if (cudaGetLastError() != cudaSuccess) return MRI_ECUDA;
  }
  return MRI_OK;
}

// Estimated FP64 work per cell-substep of a mechanism, for splitting the SMs of a
// mixed launch: about ten Newton iterations of rates (~40 flops per reaction) and
// triangular solves (2 n^2), plus one LU factorisation (2/3 n^3).
static double cell_cost(const Layout& L) {
  const double n = L.n, R = L.R;
  return 10.0 * (40.0 * R + 2.0 * n * n) + (2.0 / 3.0) * n * n * n;
}

int launch_stage_fast_batch(const mri_stage_group* groups, int ngroups, double Hs, double h, const mri_fast_opts& o,
                            int32_t* n_failed, cudaStream_t st) {
  const bool prec32 = (o.precision == MRI_PREC_FP32_LU);
  BatchArgs b{};
  int gidx[MRI_MAX_GROUPS];
  double load[MRI_MAX_GROUPS];
  int nb = 0, maxw = 1;
  size_t maxsmem = 0;
  double total = 0.0;
  for (int g = 0; g < ngroups; ++g) {
    const mri_stage_group& G = groups[g];
    if (G.ncell == 0) continue;
    const Mech& m = *reinterpret_cast<const Mech*>(G.mech);
    StageArgs& a = b.g[nb];
    int rc = fill_stage_args(a, G.y, G.p, G.ncell, G.phi, G.K, Hs, h, m, o, o.ramp, G.cell_status, G.cell_stats,
                             n_failed, false);
    if (rc != MRI_OK) return rc;
    int w, bl;
    size_t sm;
    // as many warps as one SM's shared memory holds for this mechanism
    if (!plan_launch(m.L, 1 << 30, w, bl, sm, prec32, G.K, 0, 1)) return MRI_EINVAL;
    b.warps[nb] = w;
    if (w > maxw) maxw = w;
    if (sm > maxsmem) maxsmem = sm;
    load[nb] = (double)G.ncell * cell_cost(m.L) / w;
    total += load[nb];
    gidx[nb] = g;
    ++nb;
  }
  if (nb == 0) return MRI_OK;
  // CTAs (one per SM) in proportion to each group's work per warp, at least one each and
  // no more than its cells need
  const int sms = device_sm_count();
  int blocks[MRI_MAX_GROUPS], used = 0;
  for (int i = 0; i < nb; ++i) {
    const int cap = (groups[gidx[i]].ncell + b.warps[i] - 1) / b.warps[i];
    int k = (int)std::floor(load[i] / total * (sms - nb)) + 1;
    blocks[i] = k < cap ? k : cap;
    used += blocks[i];
  }
  for (bool grew = true; used < sms && grew;) {   // hand out what rounding left, largest load first
    grew = false;
    int best = -1;
    for (int i = 0; i < nb; ++i) {
      const int cap = (groups[gidx[i]].ncell + b.warps[i] - 1) / b.warps[i];
      if (blocks[i] < cap && (best < 0 || load[i] / blocks[i] > load[best] / blocks[best])) best = i;
    }
    if (best >= 0) { blocks[best]++; used++; grew = true; }
  }
  b.ngroups = nb;
  b.block0[0] = 0;
  for (int i = 0; i < nb; ++i) b.block0[i + 1] = b.block0[i] + blocks[i];
  for (int i = 0; i < nb; ++i) {
    int rc = take_queue(*reinterpret_cast<const Mech*>(groups[gidx[i]].mech), b.g[i], st);
    if (rc != MRI_OK) return rc;
  }
  if (prec32) {
    if (!allow_full_smem((const void*)stage_fast_batch_kernel<true>)) return MRI_ECUDA;
    stage_fast_batch_kernel<true><<<b.block0[nb], maxw * 32, maxsmem, st>>>(b);
  } else {
    if (!allow_full_smem((const void*)stage_fast_batch_kernel<false>)) return MRI_ECUDA;
    stage_fast_batch_kernel<false><<<b.block0[nb], maxw * 32, maxsmem, st>>>(b);
  }
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

}  // namespace mri

// ------------------------------------------------------------------ C ABI

namespace mri {

bool fast_opts_ok(const mri_fast_opts* o) {
  return o && (o->method == MRI_SDIRK2 || o->method == MRI_SDIRK3 || (is_explicit(o->method) && !o->adaptive)) &&
         o->newton_rtol > 0 &&
         std::isfinite(o->newton_rtol) && o->newton_atol_Y >= 0 && o->newton_atol_T >= 0 &&
         std::isfinite(o->newton_atol_Y) && std::isfinite(o->newton_atol_T) && o->max_newton >= 1 &&
         o->max_newton <= 100 && (o->jac_policy == MRI_JAC_PER_SUBSTEP || o->jac_policy == MRI_JAC_LAZY) &&
         (o->precision == MRI_PREC_FP64 || o->precision == MRI_PREC_FP32_LU) &&
         o->ramp >= 0 && o->ramp <= 40 && o->warps_per_block >= 0 && o->warps_per_block <= kMaxWarps &&
         o->blocks_per_sm >= 0 && o->blocks_per_sm <= 8 && o->time_budget_s >= 0 &&
         o->time_budget_s <= 1e6 && (o->adaptive == 0 || o->adaptive == 1) &&
         (o->adaptive == 0 || (o->ctrl_rtol > 0 && std::isfinite(o->ctrl_rtol) && o->ctrl_atol_Y >= 0 &&
                               o->ctrl_atol_T >= 0 && std::isfinite(o->ctrl_atol_Y) &&
                               std::isfinite(o->ctrl_atol_T))) &&
         o->newton_safety > 0 && o->newton_safety <= 1.0 &&
         (o->schedule == MRI_SCHED_QUEUE || (o->schedule == MRI_SCHED_STATIC && o->time_budget_s == 0.0)) &&
         o->lu_variant >= MRI_LU_AUTO && o->lu_variant <= MRI_LU_INVERSE;
}

int mech_device_check(const Mech& m) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MRI_ECUDA;
  return dev == m.device ? MRI_OK : MRI_EINVAL;
}

int mri_stage_fast_checked(double* y, const double* p, int ncell, const double* phi, int K, double Hstage,
                           double h, const Mech& m, const mri_fast_opts& o, int32_t* cell_status,
                           int32_t* cell_stats, int32_t* n_failed, cudaStream_t st, bool sticky) {
  if (!fast_opts_ok(&o) || ncell < 0 || K < 0 || K > kMaxK) return MRI_EINVAL;
  if (const int rc = mech_device_check(m)) return rc;
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
  o->warps_per_block = 0;
  o->blocks_per_sm = 0;
  o->time_budget_s = 0.0;
  o->matrix_cache = nullptr;
  o->matrix_cache_bytes = 0;
  o->adaptive = 0;
  o->ctrl_rtol = 1e-6;
  o->ctrl_atol_Y = 1e-12;
  o->ctrl_atol_T = 1e-6;
  o->newton_safety = 3e-4;
  o->schedule = MRI_SCHED_QUEUE;
  o->lu_variant = MRI_LU_AUTO;
}

extern "C" size_t mri_matrix_cache_size(const mri_mech* mech, int ncell, int precision) {
  if (!mech || ncell < 0 || (precision != MRI_PREC_FP64 && precision != MRI_PREC_FP32_LU)) return 0;
  return mri::mc_stride(reinterpret_cast<const Mech*>(mech)->L, precision == MRI_PREC_FP32_LU) * (size_t)ncell;
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

extern "C" int mri_stage_fast_guided(double* y, const double* p, int ncell, const double* phi, int K, double t0,
                                     double Hstage, double h, const double* guess, int guess_steps, int start,
                                     const mri_mech* mech, const mri_fast_opts* opts, int32_t* cell_status,
                                     int32_t* cell_stats, int32_t* n_failed, int32_t* n_fallback,
                                     const int8_t* step_exp, void* stream) {
  (void)t0;
  if (!mech || !mri::fast_opts_ok(opts) || ncell < 0 || K < 0 || K > mri::kMaxK) return MRI_EINVAL;
  if (start < MRI_START_PREDICTOR || start > MRI_START_GUESS_FIRST) return MRI_EINVAL;
  if (mri::is_explicit(opts->method)) return MRI_EINVAL;     // no Newton iteration to start
  if (!(Hstage > 0) || !(h > 0) || !std::isfinite(Hstage) || !std::isfinite(h)) return MRI_EINVAL;
  if (start == MRI_START_GUESS || start == MRI_START_GUESS_FIRST) {
    double nsub = std::ceil(Hstage / h * (1.0 - 1e-12));
    if (!(nsub >= 1.0)) nsub = 1.0;
    if (ncell > 0 && (!guess || (double)guess_steps != nsub)) return MRI_EINVAL;
  }
  if (ncell > 0 && (!y || !p || (K > 0 && !phi))) return MRI_EINVAL;
  if (const int rc = mri::mech_device_check(*reinterpret_cast<const Mech*>(mech))) return rc;
  return mri::launch_stage_fast(y, p, ncell, phi, K, Hstage, h, *reinterpret_cast<const Mech*>(mech), *opts,
                                opts->ramp, cell_status, cell_stats, n_failed, static_cast<cudaStream_t>(stream),
                                false, guess, start, n_fallback, step_exp);
}

extern "C" int mri_stage_fast_batch(const mri_stage_group* groups, int ngroups, double t0, double Hstage, double h,
                                    const mri_fast_opts* opts, int32_t* n_failed, void* stream) {
  (void)t0;
  if (!groups || ngroups < 1 || ngroups > MRI_MAX_GROUPS || !mri::fast_opts_ok(opts)) return MRI_EINVAL;
  if (opts->warps_per_block != 0 || opts->blocks_per_sm > 1 || opts->time_budget_s != 0.0 || opts->matrix_cache ||
      opts->schedule != MRI_SCHED_QUEUE || mri::is_explicit(opts->method))
    return MRI_EINVAL;
  if (!(Hstage > 0) || !(h > 0) || !std::isfinite(Hstage) || !std::isfinite(h)) return MRI_EINVAL;
  for (int g = 0; g < ngroups; ++g) {
    const mri_stage_group& G = groups[g];
    if (!G.mech || G.ncell < 0 || G.K < 0 || G.K > mri::kMaxK) return MRI_EINVAL;
    if (G.ncell > 0 && (!G.y || !G.p || (G.K > 0 && !G.phi))) return MRI_EINVAL;
    if (const int rc = mri::mech_device_check(*reinterpret_cast<const Mech*>(G.mech))) return rc;
  }
  return mri::launch_stage_fast_batch(groups, ngroups, Hstage, h, *opts, n_failed, static_cast<cudaStream_t>(stream));
}

extern "C" int mri_stage_fast_shape(const mri_mech* mech, const mri_fast_opts* opts, int ncell, int K,
                                    int* warps_per_block, int* blocks, size_t* smem_bytes) {
  if (!mech || !mri::fast_opts_ok(opts) || ncell < 1 || K < 0 || K > mri::kMaxK) return MRI_EINVAL;
  const Mech* m = reinterpret_cast<const Mech*>(mech);
  int w = 0, b = 0;
  size_t s = 0;
  const bool expl = mri::is_explicit(opts->method);
  if (!mri::plan_launch(m->L, ncell, w, b, s, opts->precision == MRI_PREC_FP32_LU && !expl, K, opts->warps_per_block,
                        opts->blocks_per_sm, !expl, mri::kStageStaticSmem))
    return MRI_EINVAL;
  if (warps_per_block) *warps_per_block = w;
  if (blocks) *blocks = b;
  if (smem_bytes) *smem_bytes = s;
  return MRI_OK;
}

extern "C" int mri_fast_rhs(const double* y, const double* p, int ncell, const mri_mech* mech, double* f,
                            void* stream) {
  if (!mech || ncell < 0 || (ncell > 0 && (!y || !p || !f))) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  const Mech* m = reinterpret_cast<const Mech*>(mech);
  if (const int rc = mri::mech_device_check(*m)) return rc;
  int warps, blocks;
  size_t smem;
  if (!mri::plan_launch(m->L, ncell, warps, blocks, smem)) return MRI_EINVAL;
  if (!mri::allow_full_smem((const void*)mri::rhs_kernel)) return MRI_ECUDA;
  mri::rhs_kernel<<<blocks, warps * 32, smem, static_cast<cudaStream_t>(stream)>>>(
      y, p, ncell, f, static_cast<const unsigned char*>(m->d_table), m->L);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_fast_jac(const double* y, const double* p, int ncell, const mri_mech* mech, double* J,
                            void* stream) {
  if (!mech || ncell < 0 || (ncell > 0 && (!y || !p || !J))) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  const Mech* m = reinterpret_cast<const Mech*>(mech);
  if (const int rc = mri::mech_device_check(*m)) return rc;
  int warps, blocks;
  size_t smem;
  if (!mri::plan_launch(m->L, ncell, warps, blocks, smem)) return MRI_EINVAL;
  if (!mri::allow_full_smem((const void*)mri::jac_kernel)) return MRI_ECUDA;
  mri::jac_kernel<<<blocks, warps * 32, smem, static_cast<cudaStream_t>(stream)>>>(
      y, p, ncell, J, static_cast<const unsigned char*>(m->d_table), m->L);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

namespace mri {
// Launch of the batched one-warp-per-system test kernels (lu_kernel, inverse_kernel).
static int launch_batched_solve(void (*kern)(double*, double*, int, int, int, int32_t*), double* A, double* b,
                                int n, int nbatch, int32_t* info, void* stream) {
  if (n < 1 || n > 128 || nbatch < 0 || (nbatch > 0 && (!A || !b))) return MRI_EINVAL;
  if (nbatch == 0) return MRI_OK;
  const int ld = (n % 2 == 1) ? n : n + 1;
  const size_t per = ((size_t)round_up(n * ld, 2) + 2 * round_up(n, 2) + n) * 8;
  const int limit = device_smem_limit();
  int warps = (int)(limit / per);
  if (warps < 1) return MRI_EINVAL;
  if (warps > 8) warps = 8;
  int blocks = (nbatch + warps - 1) / warps;
  const int cap = device_sm_count() * 4;
  if (blocks > cap) blocks = cap;
  const size_t smem = per * warps;
  if (!allow_full_smem((const void*)kern)) return MRI_ECUDA;
  kern<<<blocks, warps * 32, smem, static_cast<cudaStream_t>(stream)>>>(A, b, n, ld, nbatch, info);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}
}  // namespace mri

extern "C" int mri_lu_solve_batched(double* A, double* b, int n, int nbatch, int32_t* info, void* stream) {
  return mri::launch_batched_solve(mri::lu_kernel, A, b, n, nbatch, info, stream);
}

extern "C" int mri_inverse_solve_batched(double* A, double* b, int n, int nbatch, int32_t* info, void* stream) {
  return mri::launch_batched_solve(mri::inverse_kernel, A, b, n, nbatch, info, stream);
}
