// CPU oracle of the MRI fast-partition solve (plain FP64).  TEST INFRASTRUCTURE
// ONLY: tests, the smoke check and the bench's CPU baseline use it; the CUDA
// product path never does.  See oracle.h for the method and its sources.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

namespace {

using cplx = std::complex<double>;
constexpr double R_U = 8.314462618;   // J/(mol K)
constexpr double P_ATM = 101325.0;    // Pa, standard-state pressure of K_c
constexpr double LN10 = 2.302585092994045684;

// ---------------------------------------------------------------- mechanism

struct Mech {
  int Ns = 0, R = 0, E = 0, n_eff = 0, n_troe = 0;
  std::vector<double> W, nasa, A, b, Ta, eff, troe;
  std::vector<int> elem, rtype, reac, prod, eff_row, troe_row;
};

struct Reader {
  const unsigned char* p;
  size_t n, off = 0;
  bool ok = true;
  template <class T>
  void get(std::vector<T>& v, size_t count) {
    size_t bytes = count * sizeof(T);
    if (off + bytes > n) { ok = false; return; }
    v.resize(count);
    if (bytes) std::memcpy(v.data(), p + off, bytes);
    off += bytes;
    off += (8 - off % 8) % 8;   // sections are 8-byte aligned
  }
};

bool parse(const void* blob, size_t nbytes, Mech& m) {
  if (!blob || nbytes < 40 || std::memcmp(blob, "MRIMECH1", 8) != 0) return false;
  Reader r{static_cast<const unsigned char*>(blob), nbytes, 8};
  std::vector<int32_t> hdr;
  r.get(hdr, 8);
  if (!r.ok) return false;
  m.Ns = hdr[0]; m.R = hdr[1]; m.E = hdr[2]; m.n_eff = hdr[3]; m.n_troe = hdr[4];
  if (m.Ns < 1 || m.R < 0 || m.E < 1 || m.n_eff < 0 || m.n_troe < 0) return false;
  r.get(m.W, m.Ns);
  r.get(m.nasa, 7 * (size_t)m.Ns);
  r.get(m.elem, (size_t)m.Ns * m.E);
  r.get(m.rtype, m.R);
  r.get(m.reac, 3 * (size_t)m.R);
  r.get(m.prod, 3 * (size_t)m.R);
  r.get(m.eff_row, m.R);
  r.get(m.troe_row, m.R);
  r.get(m.A, m.R);
  r.get(m.b, m.R);
  r.get(m.Ta, m.R);
  r.get(m.eff, (size_t)m.n_eff * m.Ns);
  r.get(m.troe, 7 * (size_t)m.n_troe);
  if (!r.ok) return false;
  for (int i = 0; i < m.R; ++i) {
    for (int k = 0; k < 3; ++k) {
      int a = m.reac[3 * i + k], c = m.prod[3 * i + k];
      if (a < -1 || a >= m.Ns || c < -1 || c >= m.Ns) return false;
    }
    if (m.reac[3 * i] < 0 || m.prod[3 * i] < 0) return false;
    if (m.rtype[i] < 0 || m.rtype[i] > 2) return false;
    if (m.rtype[i] != 0 && (m.eff_row[i] < 0 || m.eff_row[i] >= m.n_eff)) return false;
    if (m.rtype[i] == 2 && (m.troe_row[i] < 0 || m.troe_row[i] >= m.n_troe)) return false;
  }
  return true;
}

// ---------------------------------------------------------------- operation counts
// A double that counts the floating-point operations made on it, by category, in the
// calling thread: the oracle's own formulas evaluated once with this type give the
// algorithmic operation counts of a right-hand-side evaluation, a Jacobian, an LU
// factorisation and a solve (orc_flop_counts).  Comparisons and |x| are not counted.

struct OpCounts {
  long long add = 0, mul = 0, div = 0, exp = 0, log = 0, pow = 0;
};
thread_local OpCounts g_ops;

struct CD {
  double v = 0.0;
  CD() = default;
  CD(double x) : v(x) {}   // constants and doubles enter implicitly
};
inline CD operator+(CD a, CD b) { g_ops.add++; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { g_ops.add++; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { g_ops.mul++; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { g_ops.div++; return CD(a.v / b.v); }
inline CD operator-(CD a) { return CD(-a.v); }
inline CD& operator+=(CD& a, CD b) { a = a + b; return a; }
inline CD& operator-=(CD& a, CD b) { a = a - b; return a; }
inline CD& operator*=(CD& a, CD b) { a = a * b; return a; }
inline CD& operator/=(CD& a, CD b) { a = a / b; return a; }
inline bool operator<(CD a, CD b) { return a.v < b.v; }
inline bool operator>(CD a, CD b) { return a.v > b.v; }
inline bool operator==(CD a, CD b) { return a.v == b.v; }
inline CD exp(CD a) { g_ops.exp++; return CD(std::exp(a.v)); }
inline CD log(CD a) { g_ops.log++; return CD(std::log(a.v)); }
inline CD log10(CD a) { g_ops.log++; return CD(std::log10(a.v)); }
inline CD pow(CD a, double b) { g_ops.pow++; return CD(std::pow(a.v, b)); }
inline CD fabs(CD a) { return CD(std::fabs(a.v)); }
inline bool isfinite(CD a) { return std::isfinite(a.v); }
inline CD clamp_pos(CD x) { return x.v > 1e-300 ? x : CD(1e-300); }

// ---------------------------------------------------------------- thermodynamics
// NASA 7-coefficient polynomials (Gordon & McBride): cp/R, h/RT, s/R, g/RT = h/RT - s/R.

template <class S>
void thermo(const Mech& m, S T, S* cpR, S* hRT, S* sR, S* gRT) {
  using std::log;
  S lnT = log(T);
  for (int k = 0; k < m.Ns; ++k) {
    const double* a = &m.nasa[7 * k];
    S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    S cp = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
    S h = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    S s = a[0] * lnT + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
    if (cpR) cpR[k] = cp;
    if (hRT) hRT[k] = h;
    if (sR) sR[k] = s;
    if (gRT) gRT[k] = h - s;
  }
}

// ---------------------------------------------------------------- kinetics

inline double clamp_pos(double x) { return x > 1e-300 ? x : 1e-300; }
inline cplx clamp_pos(cplx x) { return x; }   // complex-step evaluations stay analytic

struct RateParts {   // per reaction, at (T, C)
  double kf, kr, Kc, M;
};

// third-body concentration [M] = sum_k alpha_k C_k (alpha = 1 without a row)
template <class S>
S third_body(const Mech& m, int r, const S* C) {
  S M = 0.0;
  int row = m.eff_row[r];
  for (int k = 0; k < m.Ns; ++k) M += (row >= 0 ? m.eff[(size_t)row * m.Ns + k] : 1.0) * C[k];
  return M;
}

// k_f, k_r and K_c of reaction r.  k = A T^b exp(-Ta/T); K_c = exp(-sum nu g/RT) (p_atm/(R T))^dn;
// falloff: k_f = k_inf (Pr/(1+Pr)) F with the Troe F; k_r = k_f / K_c.
template <class S>
void rate_coeffs(const Mech& m, int r, S T, const S* C, const S* gRT, S& kf, S& kr, S& Kc, S& M) {
  using std::exp;
  using std::log;
  using std::log10;
  using std::pow;
  S sumg = 0.0;
  int dn = 0;
  for (int j = 0; j < 3; ++j) {
    int a = m.reac[3 * r + j];
    if (a >= 0) { sumg -= gRT[a]; dn -= 1; }
    int c = m.prod[3 * r + j];
    if (c >= 0) { sumg += gRT[c]; dn += 1; }
  }
  Kc = exp(-sumg + double(dn) * log(P_ATM / (R_U * T)));
  S kinf = m.A[r] * pow(T, m.b[r]) * exp(-m.Ta[r] / T);
  M = (m.rtype[r] != 0) ? third_body(m, r, C) : S(0.0);
  if (m.rtype[r] == 2) {
    const double* t = &m.troe[7 * (size_t)m.troe_row[r]];
    S k0 = t[0] * pow(T, t[1]) * exp(-t[2] / T);
    S Pr = clamp_pos(k0 * M / kinf);
    S Fc = (1.0 - t[3]) * exp(-T / t[4]) + t[3] * exp(-T / t[5]) + exp(-t[6] / T);
    S logFc = log10(Fc);
    S c = -0.4 - 0.67 * logFc;
    S nn = 0.75 - 1.27 * logFc;
    S u = log10(Pr) + c;
    S f1 = u / (nn - 0.14 * u);
    S logF = logFc / (1.0 + f1 * f1);
    kf = kinf * (Pr / (1.0 + Pr)) * exp(logF * LN10);
  } else {
    kf = kinf;
  }
  kr = kf / Kc;
}

template <class S>
S prod_list(const int* list, const S* C) {
  S v = 1.0;
  for (int j = 0; j < 3; ++j)
    if (list[j] >= 0) v *= C[list[j]];
  return v;
}

// q_r = k_f prod C^nu' - k_r prod C^nu'' (times [M] for third-body reactions);
// wdot_k = sum_r (nu''_kr - nu'_kr) q_r
template <class S>
void progress(const Mech& m, S T, const S* C, const S* gRT, S* q, S* wdot) {
  for (int k = 0; k < m.Ns; ++k) wdot[k] = 0.0;
  for (int r = 0; r < m.R; ++r) {
    S kf, kr, Kc, M;
    rate_coeffs(m, r, T, C, gRT, kf, kr, Kc, M);
    S qr = kf * prod_list(&m.reac[3 * r], C) - kr * prod_list(&m.prod[3 * r], C);
    if (m.rtype[r] == 1) qr *= M;
    if (q) q[r] = qr;
    for (int j = 0; j < 3; ++j) {
      if (m.reac[3 * r + j] >= 0) wdot[m.reac[3 * r + j]] -= qr;
      if (m.prod[3 * r + j] >= 0) wdot[m.prod[3 * r + j]] += qr;
    }
  }
}

// Fast partition: dY_k/dt = wdot_k W_k / rho; dT/dt = -sum_k h_k wdot_k / (rho cp), constant p,
// rho = p / (R T sum_j Y_j/W_j), C_k = rho Y_k / W_k.
template <class S>
void fast_rhs(const Mech& m, const S* y, double p, S* f) {
  const int Ns = m.Ns;
  S T = y[Ns];
  S Ssum = 0.0;
  for (int k = 0; k < Ns; ++k) Ssum += y[k] / m.W[k];
  S rho = p / (R_U * T * Ssum);
  std::vector<S> C(Ns), cpR(Ns), hRT(Ns), gRT(Ns), wdot(Ns);
  for (int k = 0; k < Ns; ++k) C[k] = rho * y[k] / m.W[k];
  thermo<S>(m, T, cpR.data(), hRT.data(), nullptr, gRT.data());
  progress<S>(m, T, C.data(), gRT.data(), nullptr, wdot.data());
  S cpm = 0.0, Q = 0.0;
  for (int k = 0; k < Ns; ++k) {
    f[k] = wdot[k] * m.W[k] / rho;
    cpm += y[k] * cpR[k] / m.W[k];
    Q += hRT[k] * wdot[k];
  }
  f[Ns] = -T * Q / (rho * cpm);
}

// Analytic Jacobian of fast_rhs.  Derivation: q_r(C, T) differentiated term by
// term (product rule over the reactant / product lists, third-body [M], Troe F
// through x = log10 Pr and log10 Fcent, K_c through d ln K_c/dT = (sum nu h/RT - dn)/T),
// D = nu dq/dC, then the chain rule through C(Y, T) and rho(Y, T) at constant p.
template <class S>
void fast_jac(const Mech& m, const S* y, double p, S* J) {
  using std::exp;
  using std::log10;
  using std::pow;
  const int Ns = m.Ns, n = Ns + 1;
  S T = y[Ns];
  S Ssum = 0.0;
  for (int k = 0; k < Ns; ++k) Ssum += y[k] / m.W[k];
  S rho = p / (R_U * T * Ssum);
  std::vector<S> C(Ns), cpR(Ns), hRT(Ns), gRT(Ns), wdot(Ns, 0.0);
  for (int k = 0; k < Ns; ++k) C[k] = rho * y[k] / m.W[k];
  thermo<S>(m, T, cpR.data(), hRT.data(), nullptr, gRT.data());

  std::vector<S> D((size_t)Ns * Ns, 0.0), DT(Ns, 0.0);
  std::vector<S> dqdC(Ns);
  for (int r = 0; r < m.R; ++r) {
    S kf, kr, Kc, M;
    rate_coeffs<S>(m, r, T, C.data(), gRT.data(), kf, kr, Kc, M);
    const int* re = &m.reac[3 * r];
    const int* pr = &m.prod[3 * r];
    S fwd = prod_list(re, C.data()), rev = prod_list(pr, C.data());
    S sum_nu_h = 0.0;
    int dn = 0;
    for (int j = 0; j < 3; ++j) {
      if (re[j] >= 0) { sum_nu_h -= hRT[re[j]]; dn -= 1; }
      if (pr[j] >= 0) { sum_nu_h += hRT[pr[j]]; dn += 1; }
    }
    S dlnKc_dT = (sum_nu_h - dn) / T;
    S dlnkf_dT = (m.b[r] + m.Ta[r] / T) / T;
    S dlnkf_dM = 0.0;
    if (m.rtype[r] == 2) {
      const double* t = &m.troe[7 * (size_t)m.troe_row[r]];
      S kinf = m.A[r] * pow(T, m.b[r]) * exp(-m.Ta[r] / T);
      S k0 = t[0] * pow(T, t[1]) * exp(-t[2] / T);
      S Pr = clamp_pos(k0 * M / kinf);
      S dlnkinf_dT = (m.b[r] + m.Ta[r] / T) / T;
      S dlnk0_dT = (t[1] + t[2] / T) / T;
      S dlnPr_dT = dlnk0_dT - dlnkinf_dT;
      S e3 = exp(-T / t[4]), e1 = exp(-T / t[5]), e2 = exp(-t[6] / T);
      S Fc = (1.0 - t[3]) * e3 + t[3] * e1 + e2;
      S dFc_dT = -(1.0 - t[3]) / t[4] * e3 - t[3] / t[5] * e1 + t[6] / (T * T) * e2;
      S logFc = log10(Fc);
      S c = -0.4 - 0.67 * logFc, nn = 0.75 - 1.27 * logFc;
      S u = log10(Pr) + c;
      S den = nn - 0.14 * u;
      S f1 = u / den;
      S g = 1.0 + f1 * f1;
      S df1_du = nn / (den * den);      // d f1 / d x and d f1 / d c
      S df1_dnn = -u / (den * den);
      S dlogF_df1 = -logFc * 2.0 * f1 / (g * g);
      S dlogF_dx = dlogF_df1 * df1_du;
      S dlogF_dlogFc = 1.0 / g + dlogF_df1 * (df1_du * (-0.67) + df1_dnn * (-1.27));
      S dlogFc_dT = dFc_dT / (Fc * LN10);
      S dx_dT = dlnPr_dT / LN10;
      S dlnF_dT = LN10 * (dlogF_dx * dx_dT + dlogF_dlogFc * dlogFc_dT);
      dlnkf_dT = dlnkinf_dT + dlnPr_dT / (1.0 + Pr) + dlnF_dT;
      dlnkf_dM = (1.0 / M) * (1.0 / (1.0 + Pr) + dlogF_dx);
    }
    S dlnkr_dT = dlnkf_dT - dlnKc_dT;
    S base = kf * fwd - kr * rev;
    S wM = (m.rtype[r] == 1) ? M : 1.0;
    S dqdT = wM * (kf * dlnkf_dT * fwd - kr * dlnkr_dT * rev);
    // d(prod over list)/dC_l by the product rule
    std::fill(dqdC.begin(), dqdC.end(), S(0.0));
    for (int j = 0; j < 3; ++j) {
      if (re[j] >= 0) {
        S o = 1.0;
        for (int jj = 0; jj < 3; ++jj)
          if (jj != j && re[jj] >= 0) o *= C[re[jj]];
        dqdC[re[j]] += wM * kf * o;
      }
      if (pr[j] >= 0) {
        S o = 1.0;
        for (int jj = 0; jj < 3; ++jj)
          if (jj != j && pr[jj] >= 0) o *= C[pr[jj]];
        dqdC[pr[j]] -= wM * kr * o;
      }
    }
    if (m.rtype[r] != 0) {
      int row = m.eff_row[r];
      S s = (m.rtype[r] == 1) ? base : dlnkf_dM * base;
      for (int l = 0; l < Ns; ++l) dqdC[l] += m.eff[(size_t)row * Ns + l] * s;
    }
    S qr = wM * base;
    for (int j = 0; j < 3; ++j) {
      int a = re[j], c = pr[j];
      if (a >= 0) {
        wdot[a] -= qr; DT[a] -= dqdT;
        for (int l = 0; l < Ns; ++l) D[(size_t)a * Ns + l] -= dqdC[l];
      }
      if (c >= 0) {
        wdot[c] += qr; DT[c] += dqdT;
        for (int l = 0; l < Ns; ++l) D[(size_t)c * Ns + l] += dqdC[l];
      }
    }
  }
  // chain rule to (Y, T)
  std::vector<S> DC(Ns, 0.0);
  for (int k = 0; k < Ns; ++k)
    for (int l = 0; l < Ns; ++l) DC[k] += D[(size_t)k * Ns + l] * C[l];
  for (int k = 0; k < Ns; ++k) {
    for (int j = 0; j < Ns; ++j)
      J[(size_t)k * n + j] = (m.W[k] / m.W[j]) * (D[(size_t)k * Ns + j] - (DC[k] - wdot[k]) / (rho * Ssum));
    J[(size_t)k * n + Ns] = (m.W[k] / rho) * (DT[k] - (DC[k] - wdot[k]) / T);
  }
  // temperature row: f_T = -Phi Q / cpm, Phi = T/rho, Q = sum h/RT wdot, cpm = sum Y cp/R / W
  S Phi = T / rho, Q = 0.0, cpm = 0.0, dcpm_dT = 0.0;
  for (int k = 0; k < Ns; ++k) {
    const double* a = &m.nasa[7 * k];
    Q += hRT[k] * wdot[k];
    cpm += y[k] * cpR[k] / m.W[k];
    dcpm_dT += y[k] / m.W[k] * (a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T * T + 4.0 * a[4] * T * T * T);
  }
  for (int j = 0; j < Ns; ++j) {
    S dQ = 0.0;   // sum_k h/RT_k d wdot_k / dY_j
    for (int k = 0; k < Ns; ++k)
      dQ += hRT[k] * (D[(size_t)k * Ns + j] * rho / m.W[j] - DC[k] / (Ssum * m.W[j]));
    S dPhi = Phi / (Ssum * m.W[j]);
    J[(size_t)Ns * n + j] = -(dPhi * Q / cpm + Phi * dQ / cpm - Phi * Q * (cpR[j] / m.W[j]) / (cpm * cpm));
  }
  S dQdT = 0.0;
  for (int k = 0; k < Ns; ++k) dQdT += (cpR[k] - hRT[k]) / T * wdot[k] + hRT[k] * (DT[k] - DC[k] / T);
  J[(size_t)Ns * n + Ns] = -(2.0 * Phi / T * Q / cpm + Phi * dQdT / cpm - Phi * Q * dcpm_dT / (cpm * cpm));
}

void fast_jac_cs(const Mech& m, const double* y, double p, double* J) {
  const int n = m.Ns + 1;
  std::vector<cplx> yc(n), fc(n);
  for (int j = 0; j < n; ++j) {
    double hj = 1e-30 * std::max(std::fabs(y[j]), 1e-10);
    for (int i = 0; i < n; ++i) yc[i] = cplx(y[i], i == j ? hj : 0.0);
    fast_rhs<cplx>(m, yc.data(), p, fc.data());
    for (int i = 0; i < n; ++i) J[(size_t)i * n + j] = fc[i].imag() / hj;
  }
}

// ---------------------------------------------------------------- dense LU
// Doolittle LU with partial pivoting (largest |a|, ties -> lowest row index), in place.

template <class S>
int lu_factor(int n, S* A, int* piv) {
  using std::fabs;
  using std::isfinite;
  for (int k = 0; k < n; ++k) {
    int p = k;
    S best = fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      S v = fabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == S(0.0) || !isfinite(best)) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      S l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return 0;
}

template <class S>
void lu_solve(int n, const S* A, const int* piv, S* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= A[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= A[(size_t)i * n + j] * b[j];
    b[i] /= A[(size_t)i * n + i];
  }
}

// ---------------------------------------------------------------- SDIRK tableaux
// Alexander (1977): 2-stage order 2 and 3-stage order 3, both L-stable and stiffly accurate.

struct Tableau {
  int s = 0;
  double A[3][3] = {};
  double c[3] = {};
  double gamma = 0.0;
  double bhat[3] = {};   // embedded weights (one order lower) for the error estimate
  int q = 0;             // order of the estimate's leading term: the controller uses err^(-1/q)
};

Tableau sdirk(int method) {
  Tableau t;
  if (method == 2) {
    double g = 1.0 - 1.0 / std::sqrt(2.0);
    t.s = 2; t.gamma = g;
    t.A[0][0] = g;
    t.A[1][0] = 1.0 - g; t.A[1][1] = g;
    t.c[0] = g; t.c[1] = 1.0;
    // first-order embedded weights (1, 0): the estimate is h gamma (F_2 - F_1)
    t.bhat[0] = 1.0; t.bhat[1] = 0.0;
    t.q = 2;
  } else if (method == 3) {
    // gamma: the root in (0, 1) of g^3 - 3 g^2 + 3/2 g - 1/6 = 0 with L-stability (~0.4358665)
    double g = 0.4358665215;
    for (int it = 0; it < 60; ++it) {
      double fg = ((g - 3.0) * g + 1.5) * g - 1.0 / 6.0;
      double dfg = (3.0 * g - 6.0) * g + 1.5;
      g -= fg / dfg;
    }
    t.s = 3; t.gamma = g;
    t.A[0][0] = g;
    t.A[1][0] = (1.0 - g) / 2.0; t.A[1][1] = g;
    t.A[2][0] = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0;
    t.A[2][1] = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
    t.A[2][2] = g;
    t.c[0] = g; t.c[1] = (1.0 + g) / 2.0; t.c[2] = 1.0;
    // second-order embedded weights on the first two stages: sum bhat = 1 and
    // bhat . c = 1/2 with bhat_3 = 0
    t.bhat[1] = (0.5 - t.c[0]) / (t.c[1] - t.c[0]);
    t.bhat[0] = 1.0 - t.bhat[1];
    t.bhat[2] = 0.0;
    t.q = 3;
  }
  return t;
}

// ---------------------------------------------------------------- explicit fast methods
// The paper's explicit fast integrators (Sec. 3.2, the MRI-P(k) family) are classical
// explicit Runge-Kutta methods; three of them from their textbook definitions:
//   Heun (order 2):   c = (0, 1),           a21 = 1,                      b = (1/2, 1/2)
//   Kutta (order 3):  c = (0, 1/2, 1),      a21 = 1/2, a31 = -1, a32 = 2,  b = (1/6, 2/3, 1/6)
//   classical RK4:    c = (0, 1/2, 1/2, 1), a21 = a32 = 1/2, a43 = 1,      b = (1/6, 1/3, 1/3, 1/6)
// Method codes 12, 13, 14 (order + 10).

struct ErkTab {
  int s = 0;
  double A[4][4] = {};
  double b[4] = {};
  double c[4] = {};
};

bool is_erk(int method) { return method == 12 || method == 13 || method == 14; }

ErkTab erk(int method) {
  ErkTab t;
  if (method == 12) {
    t.s = 2;
    t.A[1][0] = 1.0;
    t.b[0] = 0.5; t.b[1] = 0.5;
    t.c[1] = 1.0;
  } else if (method == 13) {
    t.s = 3;
    t.A[1][0] = 0.5;
    t.A[2][0] = -1.0; t.A[2][1] = 2.0;
    t.b[0] = 1.0 / 6.0; t.b[1] = 2.0 / 3.0; t.b[2] = 1.0 / 6.0;
    t.c[1] = 0.5; t.c[2] = 1.0;
  } else if (method == 14) {
    t.s = 4;
    t.A[1][0] = 0.5;
    t.A[2][1] = 0.5;
    t.A[3][2] = 1.0;
    t.b[0] = 1.0 / 6.0; t.b[1] = 1.0 / 3.0; t.b[2] = 1.0 / 3.0; t.b[3] = 1.0 / 6.0;
    t.c[1] = 0.5; t.c[2] = 0.5; t.c[3] = 1.0;
  }
  return t;
}

// ---------------------------------------------------------------- generic stiff step

struct Problem {   // one independent unit of a fast IVP (a cell)
  int n = 0;
  std::vector<double> atol;
  virtual ~Problem() = default;
  virtual void rhs(double t, const double* y, double* f) const = 0;
  virtual void jac(double t, const double* y, double* J) const = 0;
};

struct Forcing {   // r(theta) = sum_k rhohat^k phi_k, rhohat = (theta - t0)/Hs
  const double* phi = nullptr;
  int K = 0;
};

struct StepStats { int newton = 0, jac = 0; };

double wrms(int n, const double* d, const double* z, double rtol, const double* atol) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = rtol * std::fabs(z[i]) + atol[i];
    double v = d[i] / w;
    s += v * v;
  }
  return std::sqrt(s / n);
}

// One SDIRK substep from (t, y) of size h for v' = rhs(t, v) + r(theta).  The forcing's
// normalized time rhohat = (theta - t0)/Hs of stage j is (tau + c_j h)/Hs where tau is the
// substep's offset from the start t0 of the MRI stage.  Each stage solves
//   Z_i - y - h sum_{j<i} a_ij F_j - h gamma F(t + c_i h, Z_i) = 0
// by full Newton from the previous stage value; F_i of a converged stage is taken from
// the stage equation.  Returns 0, or 1 when a stage does not converge.
int sdirk_step(const Problem& P, const Tableau& tab, double t, double h, double* y, const Forcing& fo,
               double tau, double Hs, const orc_opts& o, StepStats& st, double* err_out = nullptr) {
  const int n = P.n;
  std::vector<double> F((size_t)tab.s * n), Z(y, y + n), base(n), f(n), G(n), Mx((size_t)n * n), d(n);
  std::vector<int> piv(n);
  for (int i = 0; i < tab.s; ++i) {
    double ti = t + tab.c[i] * h;
    double rh = (tau + tab.c[i] * h) / Hs;
    std::vector<double> r(n, 0.0);
    double pw = 1.0;
    for (int k = 0; k < fo.K; ++k) {
      for (int q = 0; q < n; ++q) r[q] += pw * fo.phi[(size_t)k * n + q];
      pw *= rh;
    }
    for (int q = 0; q < n; ++q) {
      base[q] = y[q];
      for (int j = 0; j < i; ++j) base[q] += h * tab.A[i][j] * F[(size_t)j * n + q];
    }
    bool conv = false;
    for (int it = 0; it < o.max_newton; ++it) {
      P.rhs(ti, Z.data(), f.data());
      for (int q = 0; q < n; ++q) G[q] = Z[q] - base[q] - h * tab.gamma * (f[q] + r[q]);
      P.jac(ti, Z.data(), Mx.data());
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) Mx[(size_t)a * n + b] = (a == b ? 1.0 : 0.0) - h * tab.gamma * Mx[(size_t)a * n + b];
      st.jac++;
      st.newton++;
      if (lu_factor(n, Mx.data(), piv.data()) != 0) return 1;
      for (int q = 0; q < n; ++q) d[q] = -G[q];
      lu_solve(n, Mx.data(), piv.data(), d.data());
      for (int q = 0; q < n; ++q) Z[q] += d[q];
      double nd = wrms(n, d.data(), Z.data(), o.rtol, P.atol.data());
      if (!std::isfinite(nd)) return 1;
      if (nd <= 1.0) { conv = true; break; }
    }
    if (!conv) return 1;
    for (int q = 0; q < n; ++q) F[(size_t)i * n + q] = (Z[q] - base[q]) / (h * tab.gamma);
  }
  for (int q = 0; q < n; ++q) y[q] = Z[q];   // stiffly accurate: y_{n+1} = Z_s
  if (err_out) {
    // local error estimate: h sum_i (b_i - bhat_i) F_i with b_i = a_{s,i}, in the WRMS norm
    // of the controller's tolerances at the new state
    double acc = 0.0;
    for (int q = 0; q < n; ++q) {
      double e = 0.0;
      for (int i = 0; i < tab.s; ++i) e += (tab.A[tab.s - 1][i] - tab.bhat[i]) * F[(size_t)i * n + q];
      e *= h;
      const double wgt = o.ctrl_rtol * std::fabs(y[q]) + (q == n - 1 ? o.ctrl_atol_T : o.ctrl_atol_Y);
      acc += (e / wgt) * (e / wgt);
    }
    *err_out = std::sqrt(acc / n);
  }
  return 0;
}

// One explicit Runge-Kutta substep from (t, y) of size h for v' = rhs(t, v) + r(theta):
// K_i = rhs(t + c_i h, Y_i) + r(rhohat_i), Y_i = y + h sum_{j<i} a_ij K_j, with rhohat_i
// = (tau + c_i h)/Hs as in sdirk_step; y <- y + h sum_i b_i K_i.  Counts the right-hand-
// side evaluations in st.newton.  Returns 1 when the new state is not finite.
int erk_step(const Problem& P, const ErkTab& tab, double t, double h, double* y, const Forcing& fo, double tau,
             double Hs, StepStats& st) {
  const int n = P.n;
  std::vector<double> K((size_t)tab.s * n), Y(n);
  for (int i = 0; i < tab.s; ++i) {
    for (int q = 0; q < n; ++q) {
      Y[q] = y[q];
      for (int j = 0; j < i; ++j) Y[q] += h * tab.A[i][j] * K[(size_t)j * n + q];
    }
    double* Ki = &K[(size_t)i * n];
    P.rhs(t + tab.c[i] * h, Y.data(), Ki);
    st.newton++;
    const double rh = (tau + tab.c[i] * h) / Hs;
    double pw = 1.0;
    for (int k = 0; k < fo.K; ++k) {
      for (int q = 0; q < n; ++q) Ki[q] += pw * fo.phi[(size_t)k * n + q];
      pw *= rh;
    }
  }
  bool finite = true;
  for (int q = 0; q < n; ++q) {
    double inc = 0.0;
    for (int i = 0; i < tab.s; ++i) inc += tab.b[i] * K[(size_t)i * n + q];
    y[q] += h * inc;
    finite = finite && std::isfinite(y[q]);
  }
  return finite ? 0 : 1;
}

// Step-size factor of the adaptive controller: the largest of 4, 2, 1, 1/2 not above
// 0.9 err^(-1/q), else 1/4.  Powers of two keep every substep size and offset a
// dyadic multiple of the initial substep.
double ctrl_factor(double err, int q) {
  const double F[4] = {4.0, 2.0, 1.0, 0.5};
  for (int k = 0; k < 4; ++k) {
    const double th = 0.9 / F[k];
    double thq = th;
    for (int j = 1; j < q; ++j) thq *= th;
    if (err <= thq) return F[k];
  }
  return 0.25;
}

int n_substeps(double Hs, double h) {
  double r = Hs / h;
  int m = (int)std::ceil(r * (1.0 - 1e-12));
  return m < 1 ? 1 : m;
}

// Fast IVP over one MRI stage of length Hs starting at t0: n_sub uniform SDIRK substeps of
// size hh = Hs/n_sub.  With ramp = R > 0 the first substep is replaced by the start-up
// sequence hh 2^-R, hh 2^-R, hh 2^(1-R), ..., hh 2^-1 (sizes sum to hh exactly), which
// lets Newton follow a state far from the fast manifold onto it.
int fast_stage_adaptive(const Problem& P, const Tableau& tab, double t0, double Hs, double h, double* y,
                        const Forcing& fo, const orc_opts& o, int32_t* stats, int step_exp);

int fast_stage_unit(const Problem& P, const Tableau& tab, double t0, double Hs, double h, double* y,
                    const Forcing& fo, const orc_opts& o, int32_t* stats, int step_exp = 0) {
  if (o.adaptive) return fast_stage_adaptive(P, tab, t0, Hs, h, y, fo, o, stats, step_exp);
  int n_sub = n_substeps(Hs, h);
  double hh = Hs / n_sub;
  std::vector<double> tau, hs;   // substep offsets within the stage and sizes
  int R = o.ramp > 0 ? o.ramp : 0;
  if (R > 0) {
    tau.push_back(0.0);
    hs.push_back(std::ldexp(hh, -R));
    for (int k = 1; k <= R; ++k) {
      tau.push_back(std::ldexp(hh, k - 1 - R));
      hs.push_back(std::ldexp(hh, k - 1 - R));
    }
  } else {
    tau.push_back(0.0);
    hs.push_back(hh);
  }
  for (int s = 1; s < n_sub; ++s) {
    tau.push_back(s * hh);
    hs.push_back(hh);
  }
  StepStats st;
  int status = 0, done = 0;
  const bool explicit_rk = is_erk(o.method);
  const ErkTab et = explicit_rk ? erk(o.method) : ErkTab();
  for (size_t s = 0; s < hs.size(); ++s) {
    std::vector<double> save(y, y + P.n);
    const int rc = explicit_rk ? erk_step(P, et, t0 + tau[s], hs[s], y, fo, tau[s], Hs, st)
                               : sdirk_step(P, tab, t0 + tau[s], hs[s], y, fo, tau[s], Hs, o, st);
    if (rc != 0) {
      std::copy(save.begin(), save.end(), y);
      status = 1;
      break;
    }
    done++;
  }
  if (stats) {
    stats[0] += done; stats[1] += st.newton; stats[2] += st.jac; stats[3] += status;
  }
  return status;
}

// Fast IVP over one MRI stage with adaptive substeps: start from the uniform substep
// Hs/n_sub times 2^step_exp (step_exp clamped to [-20, 10]; a predicted first step);
// after each SDIRK step accept it when the embedded error estimate is at
// most 1 (next size factor from ctrl_factor), else repeat it with the factor (1/2 or
// 1/4); a step whose Newton iteration fails is repeated at 1/4 of the size.  The last
// step ends exactly at Hs; sizes never exceed Hs.  The cell fails (keeping its last
// accepted state) when a step falls below Hs 2^-40 or after 10000 attempts.
int fast_stage_adaptive(const Problem& P, const Tableau& tab, double t0, double Hs, double h, double* y,
                        const Forcing& fo, const orc_opts& o, int32_t* stats, int step_exp) {
  const int n_sub = n_substeps(Hs, h);
  double hc = std::ldexp(Hs / n_sub, std::min(10, std::max(-20, step_exp)));
  const double h_floor = std::ldexp(Hs, -40);
  double t = 0.0;
  StepStats st;
  int status = 0, done = 0, attempts = 0;
  std::vector<double> save(P.n);
  while (t < Hs) {
    if (hc < h_floor || attempts >= 10000) { status = 1; break; }
    ++attempts;
    const bool last = (t + hc >= Hs * (1.0 - 1e-12));
    const double hk = last ? Hs - t : hc;
    std::copy(y, y + P.n, save.begin());
    double err = 0.0;
    if (sdirk_step(P, tab, t0 + t, hk, y, fo, t, Hs, o, st, &err) != 0) {
      std::copy(save.begin(), save.end(), y);
      hc = hk * 0.25;
      continue;
    }
    const double fac = ctrl_factor(err, tab.q);
    if (err <= 1.0) {
      t = last ? Hs : t + hk;
      done++;
      hc = std::min(hk * fac, Hs);
    } else {
      std::copy(save.begin(), save.end(), y);
      hc = hk * fac;
    }
  }
  if (stats) {
    stats[0] += done; stats[1] += st.newton; stats[2] += st.jac; stats[3] += status;
  }
  return status;
}

// ---------------------------------------------------------------- chemistry problem

struct ChemCell : Problem {
  const Mech* m;
  double p;
  ChemCell(const Mech* mm, double pp, const orc_opts& o) : m(mm), p(pp) {
    n = mm->Ns + 1;
    atol.assign(n, o.atol_Y);
    atol[n - 1] = o.atol_T;
  }
  void rhs(double, const double* y, double* f) const override { fast_rhs<double>(*m, y, p, f); }
  void jac(double, const double* y, double* J) const override { fast_jac(*m, y, p, J); }
};

template <class Fn>
void parallel_for(int count, int nthreads, Fn fn) {
  if (nthreads <= 1 || count <= 1) {
    for (int i = 0; i < count; ++i) fn(i);
    return;
  }
  nthreads = std::min(nthreads, count);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) {
    int lo = (int)((long long)count * t / nthreads), hi = (int)((long long)count * (t + 1) / nthreads);
    th.emplace_back([=] { for (int i = lo; i < hi; ++i) fn(i); });
  }
  for (auto& x : th) x.join();
}

int stage_fast(const Mech& m, double* y, const double* p, int ncell, const double* phi, int K, double Hs,
               double h, const orc_opts& o, int32_t* status, int32_t* stats, int nthreads,
               const int8_t* step_exp = nullptr) {
  const int n = m.Ns + 1;
  Tableau tab = sdirk(o.method);
  std::vector<int> fails(ncell, 0);
  parallel_for(ncell, nthreads, [&](int c) {
    ChemCell P(&m, p[c], o);
    Forcing fo{phi ? phi + (size_t)c * K * n : nullptr, phi ? K : 0};
    int32_t* sc = stats ? stats + 4 * (size_t)c : nullptr;
    int s = fast_stage_unit(P, tab, 0.0, Hs, h, y + (size_t)c * n, fo, o, sc, step_exp ? step_exp[c] : 0);
    if (status) status[c] = s;
    fails[c] = s;
  });
  for (int c = 0; c < ncell; ++c)
    if (fails[c]) return 1;
  return 0;
}

// ---------------------------------------------------------------- slow partition
// f^S = -u . grad(y) + D lap(y), periodic central differences applied to every component.

void slow_rhs(const double* y, double* f, int n, const orc_grid& g) {
  const int N[3] = {g.nx, g.ny, g.nz};
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  for (long long c = 0; c < ncell * n; ++c) f[c] = 0.0;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long long c = ((long long)k * g.ny + j) * g.nx + i;
        int idx[3] = {i, j, k};
        for (int ax = 0; ax < 3; ++ax) {
          if (N[ax] == 1) continue;
          auto nb = [&](int off) {
            int id[3] = {idx[0], idx[1], idx[2]};
            id[ax] = ((id[ax] + off) % N[ax] + N[ax]) % N[ax];
            return ((long long)id[2] * g.ny + id[1]) * g.nx + id[0];
          };
          for (int q = 0; q < n; ++q) {
            double d1, d2;
            double f0 = y[c * n + q];
            double fp1 = y[nb(1) * n + q], fm1 = y[nb(-1) * n + q];
            if (g.order == 4) {
              double fp2 = y[nb(2) * n + q], fm2 = y[nb(-2) * n + q];
              d1 = (-fp2 + 8.0 * fp1 - 8.0 * fm1 + fm2) / (12.0 * g.dx);
              d2 = (-fp2 + 16.0 * fp1 - 30.0 * f0 + 16.0 * fm1 - fm2) / (12.0 * g.dx * g.dx);
            } else {
              d1 = (fp1 - fm1) / (2.0 * g.dx);
              d2 = (fp1 - 2.0 * f0 + fm1) / (g.dx * g.dx);
            }
            f[c * n + q] += -g.u[ax] * d1 + g.D * d2;
          }
        }
      }
}

// ---------------------------------------------------------------- MRI3 (Knoth-Wolke, MIS form)
// Base explicit RK3: c = (0, 1/3, 3/4), a21 = 1/3, a31 = -3/16, a32 = 15/16, b = (1/6, 3/10, 8/15);
// the MIS form appends b as a fourth row with c_4 = 1.

struct MriTab {
  int s = 4;
  double A[4][4] = {};
  double c[4] = {};
};

MriTab kw3() {
  MriTab t;
  t.A[1][0] = 1.0 / 3.0;
  t.A[2][0] = -3.0 / 16.0; t.A[2][1] = 15.0 / 16.0;
  t.A[3][0] = 1.0 / 6.0; t.A[3][1] = 3.0 / 10.0; t.A[3][2] = 8.0 / 15.0;
  t.c[0] = 0.0; t.c[1] = 1.0 / 3.0; t.c[2] = 3.0 / 4.0; t.c[3] = 1.0;
  return t;
}

// constant forcing of stage i: (1/dc_i) sum_j (a_ij - a_{i-1,j}) fS_j
void mis_forcing(const MriTab& t, int i, const std::vector<const double*>& fS, size_t len, double* out) {
  double dc = t.c[i] - t.c[i - 1];
  for (size_t q = 0; q < len; ++q) {
    double v = 0.0;
    for (int j = 0; j < i; ++j) v += (t.A[i][j] - t.A[i - 1][j]) * fS[j][q];
    out[q] = v / dc;
  }
}

int mri_step(const Mech& m, double* y, const double* p, const orc_grid& g, double H, double h,
             const orc_opts& o, int32_t* status, int32_t* stats, int nthreads) {
  const int n = m.Ns + 1;
  const size_t ncell = (size_t)g.nx * g.ny * g.nz, len = ncell * n;
  MriTab t = kw3();
  std::vector<std::vector<double>> fS(t.s - 1, std::vector<double>(len));
  std::vector<const double*> fp;
  std::vector<double> phi(len);
  int rc = 0;
  orc_opts oi = o;
  for (int i = 1; i < t.s; ++i) {
    slow_rhs(y, fS[i - 1].data(), n, g);   // f^S(Y_i) with Y_i the current state
    fp.push_back(fS[i - 1].data());
    mis_forcing(t, i, fp, len, phi.data());
    double Hs = (t.c[i] - t.c[i - 1]) * H;
    oi.ramp = (i == 1) ? o.ramp : 0;        // the start-up sequence belongs to the first fast stage
    rc |= stage_fast(m, y, p, (int)ncell, phi.data(), 1, Hs, h, oi, status, stats, nthreads);
  }
  return rc;
}

// ---------------------------------------------------------------- coupled single-rate reference

struct Coupled : Problem {
  const Mech* m;
  const double* p;
  orc_grid g;
  int ncell;
  Coupled(const Mech* mm, const double* pp, const orc_grid& gg, const orc_opts& o) : m(mm), p(pp), g(gg) {
    ncell = g.nx * g.ny * g.nz;
    int nc = mm->Ns + 1;
    n = ncell * nc;
    atol.resize(n);
    for (int c = 0; c < ncell; ++c) {
      for (int q = 0; q < nc - 1; ++q) atol[c * nc + q] = o.atol_Y;
      atol[c * nc + nc - 1] = o.atol_T;
    }
  }
  void rhs(double, const double* y, double* f) const override {
    int nc = m->Ns + 1;
    slow_rhs(y, f, nc, g);
    std::vector<double> ff(nc);
    for (int c = 0; c < ncell; ++c) {
      fast_rhs<double>(*m, y + (size_t)c * nc, p[c], ff.data());
      for (int q = 0; q < nc; ++q) f[(size_t)c * nc + q] += ff[q];
    }
  }
  void jac(double, const double* y, double* J) const override {
    int nc = m->Ns + 1;
    std::fill(J, J + (size_t)n * n, 0.0);
    // slow part is linear: its Jacobian columns are slow_rhs of unit vectors
    std::vector<double> e(n, 0.0), col(n);
    for (int a = 0; a < n; ++a) {
      e[a] = 1.0;
      slow_rhs(e.data(), col.data(), nc, g);
      for (int b = 0; b < n; ++b) J[(size_t)b * n + a] = col[b];
      e[a] = 0.0;
    }
    std::vector<double> Jc((size_t)nc * nc);
    for (int c = 0; c < ncell; ++c) {
      fast_jac(*m, y + (size_t)c * nc, p[c], Jc.data());
      for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) J[((size_t)c * nc + a) * n + (size_t)c * nc + b] += Jc[(size_t)a * nc + b];
    }
  }
};

// ---------------------------------------------------------------- scalar and KPR test problems

struct Scalar : Problem {
  int kind;
  double lam;
  Scalar(int k, double l) : kind(k), lam(l) { n = 1; atol.assign(1, 1e-14); }
  void rhs(double t, const double* y, double* f) const override {
    f[0] = (kind == 0) ? lam * y[0] : lam * (y[0] - std::cos(t)) - std::sin(t);
  }
  void jac(double, const double*, double* J) const override { J[0] = lam; }
};

// KPR multirate problem: u* = sqrt(3 + cos(beta t)), v* = sqrt(2 + cos(omega t));
// y' = Lambda Phi(y, t) - [beta sin(beta t)/(2u), omega sin(omega t)/(2v)],
// Phi = [(-3 + u^2 - cos(beta t))/(2u), (-2 + v^2 - cos(omega t))/(2v)], Lambda = [[G, e], [e, -1]].
// Slow partition: the u row; fast partition: the v row.
struct KPR {
  double G, e, beta, omega;
  double phiu(double t, double u) const { return (-3.0 + u * u - std::cos(beta * t)) / (2.0 * u); }
  double phiv(double t, double v) const { return (-2.0 + v * v - std::cos(omega * t)) / (2.0 * v); }
  double dphiu(double t, double u) const { return 1.0 - phiu(t, u) / u; }   // d phiu/du
  double dphiv(double t, double v) const { return 1.0 - phiv(t, v) / v; }
};

struct KPRFast : Problem {
  KPR k;
  explicit KPRFast(const KPR& kk) : k(kk) { n = 2; atol.assign(2, 1e-12); }
  void rhs(double t, const double* y, double* f) const override {
    f[0] = 0.0;
    f[1] = k.e * k.phiu(t, y[0]) - k.phiv(t, y[1]) - k.omega * std::sin(k.omega * t) / (2.0 * y[1]);
  }
  void jac(double t, const double* y, double* J) const override {
    J[0] = 0.0; J[1] = 0.0;
    J[2] = k.e * k.dphiu(t, y[0]);
    J[3] = -k.dphiv(t, y[1]) + k.omega * std::sin(k.omega * t) / (2.0 * y[1] * y[1]);
  }
};

void kpr_slow(const KPR& k, double t, const double* y, double* f) {
  f[0] = k.G * k.phiu(t, y[0]) + k.e * k.phiv(t, y[1]) - k.beta * std::sin(k.beta * t) / (2.0 * y[0]);
  f[1] = 0.0;
}

}  // namespace

// =============================================================== C ABI

extern "C" {

void* orc_mech_load(const void* blob, size_t nbytes) {
  Mech* m = new Mech;
  if (!parse(blob, nbytes, *m)) { delete m; return nullptr; }
  return m;
}

void orc_mech_free(void* mech) { delete static_cast<Mech*>(mech); }

int orc_mech_info(const void* mech, int* ns, int* nr) {
  if (!mech) return -1;
  const Mech* m = static_cast<const Mech*>(mech);
  if (ns) *ns = m->Ns;
  if (nr) *nr = m->R;
  return 0;
}

int orc_thermo(const void* mech, double T, double* cpR, double* hRT, double* sR, double* gRT) {
  if (!mech || !(T > 0)) return -1;
  thermo<double>(*static_cast<const Mech*>(mech), T, cpR, hRT, sR, gRT);
  return 0;
}

int orc_rate_coeffs(const void* mech, double T, const double* C, double* kf, double* kr, double* Kc) {
  if (!mech || !(T > 0)) return -1;
  const Mech& m = *static_cast<const Mech*>(mech);
  std::vector<double> g(m.Ns);
  thermo<double>(m, T, nullptr, nullptr, nullptr, g.data());
  for (int r = 0; r < m.R; ++r) {
    double a, b, c, M;
    rate_coeffs<double>(m, r, T, C, g.data(), a, b, c, M);
    if (kf) kf[r] = a;
    if (kr) kr[r] = b;
    if (Kc) Kc[r] = c;
  }
  return 0;
}

int orc_progress(const void* mech, double T, const double* C, double* q, double* wdot) {
  if (!mech || !(T > 0)) return -1;
  const Mech& m = *static_cast<const Mech*>(mech);
  std::vector<double> g(m.Ns);
  thermo<double>(m, T, nullptr, nullptr, nullptr, g.data());
  progress<double>(m, T, C, g.data(), q, wdot);
  return 0;
}

int orc_rhs(const void* mech, const double* y, double p, double* f) {
  if (!mech) return -1;
  fast_rhs<double>(*static_cast<const Mech*>(mech), y, p, f);
  return 0;
}

int orc_jac(const void* mech, const double* y, double p, double* J) {
  if (!mech) return -1;
  fast_jac(*static_cast<const Mech*>(mech), y, p, J);
  return 0;
}

int orc_jac_cs(const void* mech, const double* y, double p, double* J) {
  if (!mech) return -1;
  fast_jac_cs(*static_cast<const Mech*>(mech), y, p, J);
  return 0;
}

int orc_flop_counts(const void* mech, const double* y, double p, double hg, long long* out) {
  if (!mech || !y || !out || !(p > 0) || !(hg > 0)) return -1;
  const Mech& m = *static_cast<const Mech*>(mech);
  const int n = m.Ns + 1;
  auto take = [&](int row) {
    const long long v[6] = {g_ops.add, g_ops.mul, g_ops.div, g_ops.exp, g_ops.log, g_ops.pow};
    for (int c = 0; c < 6; ++c) out[row * 6 + c] = v[c];
    g_ops = OpCounts();
  };
  std::vector<CD> yc(y, y + n), f(n), Jc((size_t)n * n);
  g_ops = OpCounts();
  fast_rhs<CD>(m, yc.data(), p, f.data());
  take(0);
  fast_jac<CD>(m, yc.data(), p, Jc.data());
  take(1);
  // LU of the Newton matrix I - hg J at this state (pivots as in the solver)
  std::vector<double> J((size_t)n * n);
  fast_jac<double>(m, y, p, J.data());
  std::vector<CD> M((size_t)n * n), b(n, CD(1.0));
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) M[(size_t)a * n + c] = CD((a == c ? 1.0 : 0.0) - hg * J[(size_t)a * n + c]);
  std::vector<int> piv(n);
  g_ops = OpCounts();
  if (lu_factor<CD>(n, M.data(), piv.data()) != 0) return 1;
  take(2);
  lu_solve<CD>(n, M.data(), piv.data(), b.data());
  take(3);
  return 0;
}

int orc_lu_solve(int n, double* A, int* piv, double* b) {
  if (n < 1) return -1;
  int rc = lu_factor(n, A, piv);
  if (rc) return rc;
  lu_solve(n, A, piv, b);
  return 0;
}

int orc_sdirk_tableau(int method, double* A, double* b, double* c, int* s) {
  if (method != 2 && method != 3) return -1;
  Tableau t = sdirk(method);
  *s = t.s;
  for (int i = 0; i < t.s; ++i) {
    c[i] = t.c[i];
    b[i] = t.A[t.s - 1][i];
    for (int j = 0; j < t.s; ++j) A[i * t.s + j] = t.A[i][j];
  }
  return 0;
}

int orc_sdirk_embedded(int method, double* bhat, int* q) {
  if (method != 2 && method != 3) return -1;
  Tableau t = sdirk(method);
  for (int i = 0; i < t.s; ++i) bhat[i] = t.bhat[i];
  *q = t.q;
  return 0;
}

int orc_erk_tableau(int method, double* A, double* b, double* c, int* s) {
  if (!is_erk(method)) return -1;
  ErkTab t = erk(method);
  *s = t.s;
  for (int i = 0; i < t.s; ++i) {
    c[i] = t.c[i];
    b[i] = t.b[i];
    for (int j = 0; j < t.s; ++j) A[i * t.s + j] = t.A[i][j];
  }
  return 0;
}

int orc_erk_scalar(int method, int problem, double lam, double t0, double t1, int nsteps, double y0,
                   double* y_out) {
  if (!is_erk(method) || nsteps < 1) return -1;
  Scalar P(problem, lam);
  ErkTab tab = erk(method);
  double y = y0, hh = (t1 - t0) / nsteps;
  StepStats st;
  Forcing none;
  for (int s = 0; s < nsteps; ++s)
    if (erk_step(P, tab, t0 + s * hh, hh, &y, none, s * hh, t1 - t0, st) != 0) return 1;
  *y_out = y;
  return 0;
}

int orc_mri_tableau(double* A, double* c, int* s) {
  MriTab t = kw3();
  *s = t.s;
  for (int i = 0; i < t.s; ++i) {
    c[i] = t.c[i];
    for (int j = 0; j < t.s; ++j) A[i * t.s + j] = t.A[i][j];
  }
  return 0;
}

int orc_mri_coupling(double* G, int* s) {
  MriTab t = kw3();
  *s = t.s;
  for (int i = 0; i < t.s * t.s; ++i) G[i] = 0.0;
  for (int i = 1; i < t.s; ++i)
    for (int j = 0; j < i; ++j) G[i * t.s + j] = (t.A[i][j] - t.A[i - 1][j]) / (t.c[i] - t.c[i - 1]);
  return 0;
}

int orc_stage_fast(const void* mech, double* y, const double* p, int ncell, const double* phi, int K,
                   double Hs, double h, const orc_opts* o, int32_t* status, int32_t* stats, int nthreads) {
  if (!mech || !o || ncell < 0 || K < 0 || !(Hs > 0) || !(h > 0)) return -1;
  if (o->method != 2 && o->method != 3 && !(is_erk(o->method) && !o->adaptive)) return -1;
  return stage_fast(*static_cast<const Mech*>(mech), y, p, ncell, phi, K, Hs, h, *o, status, stats, nthreads);
}

int orc_stage_fast_exp(const void* mech, double* y, const double* p, int ncell, const double* phi, int K,
                       double Hs, double h, const orc_opts* o, const int8_t* step_exp, int32_t* status,
                       int32_t* stats, int nthreads) {
  if (!mech || !o || ncell < 0 || K < 0 || !(Hs > 0) || !(h > 0)) return -1;
  if (o->method != 2 && o->method != 3 && !(is_erk(o->method) && !o->adaptive)) return -1;
  return stage_fast(*static_cast<const Mech*>(mech), y, p, ncell, phi, K, Hs, h, *o, status, stats, nthreads,
                    step_exp);
}

int orc_slow_rhs(const double* y, double* f, int n, const orc_grid* g) {
  if (!g || n < 1 || g->nx < 1 || g->ny < 1 || g->nz < 1) return -1;
  slow_rhs(y, f, n, *g);
  return 0;
}

int orc_mri_step(const void* mech, double* y, const double* p, const orc_grid* g, double H, double h,
                 const orc_opts* o, int32_t* status, int32_t* stats, int nthreads) {
  if (!mech || !g || !o || !(H > 0) || !(h > 0)) return -1;
  return mri_step(*static_cast<const Mech*>(mech), y, p, *g, H, h, *o, status, stats, nthreads);
}

int orc_single_rate(const void* mech, double* y, const double* p, const orc_grid* g, double t_end,
                    int nsteps, const orc_opts* o) {
  if (!mech || !g || !o || nsteps < 1) return -1;
  Coupled P(static_cast<const Mech*>(mech), p, *g, *o);
  Tableau tab = sdirk(o->method);
  double hh = t_end / nsteps;
  StepStats st;
  Forcing none;
  for (int s = 0; s < nsteps; ++s)
    if (sdirk_step(P, tab, s * hh, hh, y, none, s * hh, t_end, *o, st) != 0) return 1;
  return 0;
}

int orc_sdirk_scalar(int method, int problem, double lam, double t0, double t1, int nsteps, double y0,
                     double* y_out) {
  if ((method != 2 && method != 3) || nsteps < 1) return -1;
  Scalar P(problem, lam);
  Tableau tab = sdirk(method);
  orc_opts o{method, 1e-14, 0.0, 0.0, 50, 0};
  double y = y0, hh = (t1 - t0) / nsteps;
  StepStats st;
  Forcing none;
  for (int s = 0; s < nsteps; ++s)
    if (sdirk_step(P, tab, t0 + s * hh, hh, &y, none, s * hh, t1 - t0, o, st) != 0) return 1;
  *y_out = y;
  return 0;
}

int orc_kpr_mri(int fast_method, double G, double e, double beta, double omega, double t1, int nsteps,
                int m_fast, double* err, double* y_out) {
  if ((fast_method != 2 && fast_method != 3 && !is_erk(fast_method)) || nsteps < 1 || m_fast < 1) return -1;
  KPR k{G, e, beta, omega};
  KPRFast P(k);
  Tableau tab = sdirk(fast_method);
  MriTab t = kw3();
  orc_opts o{fast_method, 1e-13, 0.0, 0.0, 50, 0};
  double y[2] = {std::sqrt(4.0), std::sqrt(3.0)};   // exact values at t = 0
  double H = t1 / nsteps, hfast = H / m_fast;
  for (int s = 0; s < nsteps; ++s) {
    double tn = s * H;
    std::vector<std::vector<double>> fS(t.s - 1, std::vector<double>(2));
    std::vector<const double*> fp;
    double phi[2];
    for (int i = 1; i < t.s; ++i) {
      kpr_slow(k, tn + t.c[i - 1] * H, y, fS[i - 1].data());
      fp.push_back(fS[i - 1].data());
      mis_forcing(t, i, fp, 2, phi);
      Forcing fo{phi, 1};
      double Hs = (t.c[i] - t.c[i - 1]) * H;
      if (fast_stage_unit(P, tab, tn + t.c[i - 1] * H, Hs, hfast, y, fo, o, nullptr) != 0) return 1;
    }
  }
  double ue = std::sqrt(3.0 + std::cos(beta * t1)), ve = std::sqrt(2.0 + std::cos(omega * t1));
  *err = std::max(std::fabs(y[0] - ue), std::fabs(y[1] - ve));
  if (y_out) { y_out[0] = y[0]; y_out[1] = y[1]; }
  return 0;
}

}  // extern "C"
