// Mechanism loading: parse the "MRIMECH1" blob and build the device table
// that the kernels stage into shared memory (layout in internal.cuh).
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "fastmath.cuh"
#include "internal.cuh"
#include "../../include/mri_probe.h"

namespace mri {
namespace {

struct Blob {
  int Ns = 0, R = 0, E = 0, n_eff = 0, n_troe = 0;
  std::vector<double> W, nasa, A, b, Ta, eff, troe;
  std::vector<int32_t> elem, rtype, reac, prod, eff_row, troe_row;
};

class Cursor {
 public:
  Cursor(const unsigned char* p, size_t n) : p_(p), n_(n) {}
  template <class T>
  bool take(std::vector<T>& out, size_t count) {
    size_t bytes = count * sizeof(T);
    if (pos_ + bytes > n_) return false;
    out.resize(count);
    if (bytes) std::memcpy(out.data(), p_ + pos_, bytes);
    pos_ = (pos_ + bytes + 7) & ~size_t(7);
    return true;
  }
  void seek(size_t p) { pos_ = p; }

 private:
  const unsigned char* p_;
  size_t n_, pos_ = 0;
};

bool read_blob(const void* data, size_t nbytes, Blob& B) {
  if (data == nullptr || nbytes < 40) return false;
  const unsigned char* p = static_cast<const unsigned char*>(data);
  static const char magic[8] = {'M', 'R', 'I', 'M', 'E', 'C', 'H', '1'};
  if (std::memcmp(p, magic, 8) != 0) return false;
  Cursor c(p, nbytes);
  c.seek(8);
  std::vector<int32_t> h;
  if (!c.take(h, 8)) return false;
  B.Ns = h[0]; B.R = h[1]; B.E = h[2]; B.n_eff = h[3]; B.n_troe = h[4];
  if (B.Ns < 1 || B.Ns > kMaxSpecies || B.R < 0 || B.R > kMaxReactions || B.E < 1 || B.E > 64) return false;
  if (B.n_eff < 0 || B.n_eff > B.R || B.n_troe < 0 || B.n_troe > B.R) return false;
  bool ok = c.take(B.W, B.Ns) && c.take(B.nasa, 7 * B.Ns) && c.take(B.elem, B.Ns * B.E) &&
            c.take(B.rtype, B.R) && c.take(B.reac, 3 * B.R) && c.take(B.prod, 3 * B.R) &&
            c.take(B.eff_row, B.R) && c.take(B.troe_row, B.R) && c.take(B.A, B.R) && c.take(B.b, B.R) &&
            c.take(B.Ta, B.R) && c.take(B.eff, (size_t)B.n_eff * B.Ns) && c.take(B.troe, 7 * (size_t)B.n_troe);
  if (!ok) return false;
  for (int k = 0; k < B.Ns; ++k)
    if (!(B.W[k] > 0) || !std::isfinite(B.W[k])) return false;
  for (double v : B.nasa)
    if (!std::isfinite(v)) return false;
  for (int r = 0; r < B.R; ++r) {
    if (B.rtype[r] < 0 || B.rtype[r] > 2) return false;
    if (B.reac[3 * r] < 0 || B.prod[3 * r] < 0) return false;
    for (int j = 0; j < 3; ++j)
      if (B.reac[3 * r + j] < -1 || B.reac[3 * r + j] >= B.Ns || B.prod[3 * r + j] < -1 ||
          B.prod[3 * r + j] >= B.Ns)
        return false;
    if (B.rtype[r] != 0 && (B.eff_row[r] < 0 || B.eff_row[r] >= B.n_eff)) return false;
    if (B.rtype[r] == 2 && (B.troe_row[r] < 0 || B.troe_row[r] >= B.n_troe)) return false;
    if (!(B.A[r] > 0) || !std::isfinite(B.b[r]) || !std::isfinite(B.Ta[r])) return false;
  }
  for (int t = 0; t < B.n_troe; ++t) {
    const double* q = &B.troe[7 * t];
    if (!(q[0] > 0) || !(q[4] > 0) || !(q[5] > 0) || !std::isfinite(q[6])) return false;
  }
  return true;
}

// little builder of 16-byte aligned sections
struct Sections {
  std::vector<unsigned char> buf;
  int add(size_t bytes) {
    size_t off = (buf.size() + 15) & ~size_t(15);
    buf.resize(off + ((bytes + 15) & ~size_t(15)), 0);
    return (int)off;
  }
  template <class T>
  T* at(int off) { return reinterpret_cast<T*>(buf.data() + off); }
};

// Reactions reordered so that falloff reactions come first, then third-body
// reactions, then plain ones (stable within each class).  A warp evaluates 32
// consecutive reactions per pass, so the long falloff branch runs in as few
// passes as possible instead of diverging in every pass.
Blob group_reactions(const Blob& B) {
  Blob P = B;
  std::vector<int> order;
  for (int cls : {2, 1, 0})
    for (int r = 0; r < B.R; ++r)
      if (B.rtype[r] == cls) order.push_back(r);
  for (int i = 0; i < B.R; ++i) {
    const int r = order[i];
    P.rtype[i] = B.rtype[r];
    P.eff_row[i] = B.eff_row[r];
    P.troe_row[i] = B.troe_row[r];
    P.A[i] = B.A[r];
    P.b[i] = B.b[r];
    P.Ta[i] = B.Ta[r];
    for (int j = 0; j < 3; ++j) {
      P.reac[3 * i + j] = B.reac[3 * r + j];
      P.prod[3 * i + j] = B.prod[3 * r + j];
    }
  }
  return P;
}

}  // namespace

int build_table(const Blob& Bin, Layout& L, std::vector<unsigned char>& out) {
  const Blob B = group_reactions(Bin);
  L = Layout{};
  L.Ns = B.Ns; L.R = B.R; L.n = B.Ns + 1; L.n_eff = B.n_eff; L.n_troe = B.n_troe;
  L.nsv = round_up(B.Ns + 1, 2);
  L.rv = round_up(B.R > 0 ? B.R : 1, 2);
  const int Ns = B.Ns, R = B.R, nsv = L.nsv, rv = L.rv;
  Sections S;
  L.o_cp = S.add(5 * nsv * 8);
  L.o_h = S.add(5 * nsv * 8);
  L.o_s = S.add(5 * nsv * 8);
  L.o_h5 = S.add(nsv * 8);
  L.o_s6 = S.add(nsv * 8);
  L.o_dcp = S.add(4 * nsv * 8);
  L.o_W = S.add(nsv * 8);
  L.o_invW = S.add(nsv * 8);
  L.o_lnA = S.add(rv * 8);
  L.o_b = S.add(rv * 8);
  L.o_Ta = S.add(rv * 8);
  L.o_rxn = S.add(rv * 8);
  L.o_rrow = S.add(rv * 4);
  // sparse (alpha - 1) entries
  std::vector<int> eptr(B.n_eff + 1, 0), eidx;
  std::vector<double> evals;
  for (int e = 0; e < B.n_eff; ++e) {
    for (int k = 0; k < Ns; ++k) {
      double a = B.eff[(size_t)e * Ns + k];
      if (a != 1.0) { eidx.push_back(k); evals.push_back(a - 1.0); }
    }
    eptr[e + 1] = (int)eidx.size();
  }
  L.o_eptr = S.add((B.n_eff + 1) * 4);
  L.o_eidx = S.add((eidx.size() + 1) * 4);
  L.o_eval = S.add((evals.size() + 1) * 8);
  L.o_troe = S.add((size_t)(B.n_troe > 0 ? B.n_troe : 1) * 8 * 8);

  // net stoichiometry per reaction
  std::vector<std::map<int, int>> net(R);
  for (int r = 0; r < R; ++r)
    for (int j = 0; j < 3; ++j) {
      if (B.reac[3 * r + j] >= 0) net[r][B.reac[3 * r + j]] -= 1;
      if (B.prod[3 * r + j] >= 0) net[r][B.prod[3 * r + j]] += 1;
    }
  // species -> (r, nu) lists
  std::vector<std::vector<int32_t>> wl(Ns);
  for (int r = 0; r < R; ++r)
    for (auto& kv : net[r])
      if (kv.second != 0) wl[kv.first].push_back((int32_t)(r | ((uint32_t)(kv.second & 0xffff) << 16)));
  size_t nw = 0;
  for (auto& v : wl) nw += v.size();
  // balanced production-rate sums: the species-major (species, reaction, nu) list cut
  // into 32 equal chunks, one per lane; each run of one species inside a chunk ends
  // in a partial-sum slot, and every species sums its slots
  const int gL = (int)((nw + 31) / 32);
  std::vector<int32_t> gent(nw > 0 ? nw : 1, 0);
  std::vector<std::vector<int32_t>> spslots(Ns);
  int nslot = 0;
  {
    std::vector<std::pair<int, int32_t>> flat;   // (species, packed r | nu)
    for (int k = 0; k < Ns; ++k)
      for (int32_t v : wl[k]) flat.push_back({k, v});
    for (size_t e = 0; e < flat.size(); ++e) {
      const int k = flat[e].first;
      const int r = flat[e].second & 0xffff;
      const int nu = (int)(int16_t)((uint32_t)flat[e].second >> 16);
      const bool chunk_end = ((e + 1) % gL == 0) || (e + 1 == flat.size());
      const bool last = chunk_end || flat[e + 1].first != k;
      if (e == 0 || e % gL == 0 || flat[e - 1].first != k) {   // first entry of a run
        spslots[k].push_back(nslot);
      }
      const int slot = spslots[k].back();
      if (last) ++nslot;
      gent[e] = (int32_t)(r | ((nu + 8) << 10) | (slot << 14) | ((last ? 1 : 0) << 22));
    }
  }
  if (nslot > 255) return MRI_EINVAL;   // slot field is 8 bits wide
  L.g_chunk = gL;
  L.n_went = (int)nw;
  L.n_slots = nslot;
  L.o_gent = S.add(gent.size() * 4);
  L.o_gsptr = S.add((Ns + 1) * 4);
  size_t nss = 0;
  for (auto& v : spslots) nss += v.size();
  L.o_gslot = S.add((nss + 1) * 4);
  // Jacobian column entries: species l that appears among the reactants or products of r
  std::vector<std::vector<uint64_t>> cl(Ns);
  for (int r = 0; r < R; ++r) {
    std::map<int, int> seen;
    for (int j = 0; j < 3; ++j) {
      if (B.reac[3 * r + j] >= 0) seen[B.reac[3 * r + j]] |= 1;
      if (B.prod[3 * r + j] >= 0) seen[B.prod[3 * r + j]] |= 2;
    }
    for (auto& kv : seen) {
      int l = kv.first;
      // multiplicity of l among the reactants / products, and the partners left
      // after removing one occurrence of l (d/dC_l of C_l^m X = m C_l^(m-1) X)
      int mf = 0, mr = 0;
      for (int j = 0; j < 3; ++j) {
        if (B.reac[3 * r + j] == l) mf++;
        if (B.prod[3 * r + j] == l) mr++;
      }
      int ofw[3] = {Ns, Ns, Ns}, orv[3] = {Ns, Ns, Ns};
      if (mf > 0) {
        bool removed = false;
        int nf = 0;
        for (int j = 0; j < 3; ++j) {
          int s = B.reac[3 * r + j];
          if (s < 0) continue;
          if (s == l && !removed) { removed = true; continue; }
          ofw[nf++] = s;
        }
      }
      if (mr > 0) {
        bool removed = false;
        int nr = 0;
        for (int j = 0; j < 3; ++j) {
          int s = B.prod[3 * r + j];
          if (s < 0) continue;
          if (s == l && !removed) { removed = true; continue; }
          orv[nr++] = s;
        }
      }
      uint64_t e = (uint64_t)r | ((uint64_t)mf << 16) | ((uint64_t)mr << 20) | ((uint64_t)ofw[0] << 24) |
                   ((uint64_t)ofw[1] << 32) | ((uint64_t)orv[0] << 40) | ((uint64_t)orv[1] << 48);
      cl[l].push_back(e);
    }
  }
  size_t nc = 0;
  for (auto& v : cl) nc += v.size();
  L.o_cptr = S.add((Ns + 1) * 4);
  L.o_cent = S.add((nc + 1) * 8);
  L.o_rsp = S.add((size_t)rv * 16);
  std::vector<int32_t> tbl;
  for (int r = 0; r < R; ++r)
    if (B.rtype[r] != 0) tbl.push_back(r);
  L.n_tb = (int)tbl.size();
  L.o_tbl = S.add((tbl.size() + 1) * 4);
  // per Jacobian column l: the third-body reactions r whose efficiency of species l
  // differs from 1, with alpha_rl - 1 (the part of d[M]/dC_l beyond the common 1)
  std::vector<std::vector<std::pair<int, double>>> tcl(Ns);
  for (int r : tbl)
    for (int l = 0; l < Ns; ++l) {
      const double a = B.eff[(size_t)B.eff_row[r] * Ns + l];
      if (a != 1.0) tcl[l].push_back({r, a - 1.0});
    }
  size_t ntc = 0;
  for (auto& v : tcl) ntc += v.size();
  L.o_tcptr = S.add((Ns + 1) * 4);
  L.o_tcr = S.add((ntc + 1) * 4);
  L.o_tcv = S.add((ntc + 1) * 8);
  L.o_tcv32 = S.add((ntc + 1) * 4);
  L.o_trx = S.add((size_t)(B.n_troe > 0 ? B.n_troe : 1) * 4);
  L.o_exp2 = S.add(kExpTab * 8);
  L.o_logt = S.add(kLogTabDoubles * 8);
  L.o_nu = S.add(8 * 8);
  L.o_nu32 = S.add(8 * 4);
  L.o_W32 = S.add(nsv * 4);
  L.o_invW32 = S.add(nsv * 4);
  L.o_dcp32 = S.add(4 * nsv * 4);
  L.bytes = (int)((S.buf.size() + 15) & ~size_t(15));
  S.buf.resize(L.bytes, 0);

  // ---- fill
  double* cp = S.at<double>(L.o_cp);
  double* hh = S.at<double>(L.o_h);
  double* ss = S.at<double>(L.o_s);
  double* h5 = S.at<double>(L.o_h5);
  double* s6 = S.at<double>(L.o_s6);
  double* dcp = S.at<double>(L.o_dcp);
  double* W = S.at<double>(L.o_W);
  double* invW = S.at<double>(L.o_invW);
  for (int k = 0; k < Ns; ++k) {
    const double* a = &B.nasa[7 * k];
    // cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4 (Horner coefficients)
    // h/RT = a1 + a2/2 T + a3/3 T^2 + a4/4 T^3 + a5/5 T^4 + a6 / T
    // s/R  = a1 ln T + a2 T + a3/2 T^2 + a4/3 T^3 + a5/4 T^4 + a7
    for (int j = 0; j < 5; ++j) {
      cp[j * nsv + k] = a[j];
      hh[j * nsv + k] = a[j] / (double)(j + 1);
      ss[j * nsv + k] = (j == 0) ? a[0] : a[j] / (double)j;
    }
    h5[k] = a[5];
    s6[k] = a[6];
    for (int j = 0; j < 4; ++j) dcp[j * nsv + k] = a[j + 1] * (double)(j + 1);
    W[k] = B.W[k];
    invW[k] = 1.0 / B.W[k];
  }
  double* lnA = S.at<double>(L.o_lnA);
  double* bb = S.at<double>(L.o_b);
  double* Ta = S.at<double>(L.o_Ta);
  uint64_t* rxn = S.at<uint64_t>(L.o_rxn);
  int32_t* rrow = S.at<int32_t>(L.o_rrow);
  uint64_t* rsp = S.at<uint64_t>(L.o_rsp);
  for (int r = 0; r < R; ++r) {
    lnA[r] = std::log(B.A[r]);
    bb[r] = B.b[r];
    Ta[r] = B.Ta[r];
    uint64_t w = 0;
    int dn = 0;
    for (int j = 0; j < 3; ++j) {
      int a = B.reac[3 * r + j], c = B.prod[3 * r + j];
      if (a >= 0) dn--;
      if (c >= 0) dn++;
      w |= (uint64_t)(a >= 0 ? a : Ns) << (8 * j);
      w |= (uint64_t)(c >= 0 ? c : Ns) << (8 * (3 + j));
    }
    w |= (uint64_t)(uint8_t)(int8_t)dn << 48;
    w |= (uint64_t)B.rtype[r] << 56;
    rxn[r] = w;
    uint32_t er = (B.rtype[r] != 0) ? (uint32_t)B.eff_row[r] : 0xffffu;
    uint32_t tr = (B.rtype[r] == 2) ? (uint32_t)B.troe_row[r] : 0xffffu;
    rrow[r] = (int32_t)(er | (tr << 16));
    uint64_t w0 = 0, w1 = 0;
    int cnt = 0;
    for (auto& kv : net[r]) {
      if (kv.second == 0) continue;
      w0 |= (uint64_t)kv.first << (8 * cnt);
      w1 |= (uint64_t)(uint8_t)(int8_t)kv.second << (8 * cnt);
      cnt++;
    }
    w0 |= (uint64_t)cnt << 48;
    rsp[2 * r] = w0;
    rsp[2 * r + 1] = w1;
  }
  int32_t* ep = S.at<int32_t>(L.o_eptr);
  for (int e = 0; e <= B.n_eff; ++e) ep[e] = eptr[e];
  int32_t* ei = S.at<int32_t>(L.o_eidx);
  double* ev = S.at<double>(L.o_eval);
  for (size_t i = 0; i < eidx.size(); ++i) { ei[i] = eidx[i]; ev[i] = evals[i]; }
  double* tro = S.at<double>(L.o_troe);
  for (int t = 0; t < B.n_troe; ++t) {
    const double* q = &B.troe[7 * t];
    tro[8 * t + 0] = std::log(q[0]);
    tro[8 * t + 1] = q[1];
    tro[8 * t + 2] = q[2];
    tro[8 * t + 3] = q[3];
    tro[8 * t + 4] = 1.0 / q[4];
    tro[8 * t + 5] = 1.0 / q[5];
    tro[8 * t + 6] = q[6];
    tro[8 * t + 7] = 0.0;
  }
  int pos = 0;
  {
    int32_t* ge = S.at<int32_t>(L.o_gent);
    for (size_t e = 0; e < gent.size(); ++e) ge[e] = gent[e];
    int32_t* gp = S.at<int32_t>(L.o_gsptr);
    int32_t* gs = S.at<int32_t>(L.o_gslot);
    int q = 0;
    for (int k = 0; k < Ns; ++k) {
      gp[k] = q;
      for (int32_t s : spslots[k]) gs[q++] = s;
    }
    gp[Ns] = q;
  }
  int32_t* cptr = S.at<int32_t>(L.o_cptr);
  uint64_t* cent = S.at<uint64_t>(L.o_cent);
  pos = 0;
  for (int l = 0; l < Ns; ++l) {
    cptr[l] = pos;
    for (uint64_t v : cl[l]) cent[pos++] = v;
  }
  cptr[Ns] = pos;
  int32_t* tb = S.at<int32_t>(L.o_tbl);
  for (size_t i = 0; i < tbl.size(); ++i) tb[i] = tbl[i];
  {
    int32_t* tcp = S.at<int32_t>(L.o_tcptr);
    int32_t* tcr = S.at<int32_t>(L.o_tcr);
    double* tcv = S.at<double>(L.o_tcv);
    float* tcv32 = S.at<float>(L.o_tcv32);
    int q = 0;
    for (int l = 0; l < Ns; ++l) {
      tcp[l] = q;
      for (auto& pr : tcl[l]) { tcr[q] = pr.first; tcv[q] = pr.second; tcv32[q] = (float)pr.second; ++q; }
    }
    tcp[Ns] = q;
  }
  int32_t* trx = S.at<int32_t>(L.o_trx);
  for (int r = 0; r < R; ++r)
    if (B.rtype[r] == 2) trx[B.troe_row[r]] = r;
  fill_exp_table(S.at<double>(L.o_exp2));
  fill_log_table(S.at<double>(L.o_logt));
  double* nu = S.at<double>(L.o_nu);
  for (int i = 0; i < 8; ++i) nu[i] = (double)(i - 3);
  float* nu32 = S.at<float>(L.o_nu32);
  for (int i = 0; i < 8; ++i) nu32[i] = (float)(i - 3);
  float* W32 = S.at<float>(L.o_W32);
  float* invW32 = S.at<float>(L.o_invW32);
  float* dcp32 = S.at<float>(L.o_dcp32);
  for (int k = 0; k < nsv; ++k) { W32[k] = (float)W[k]; invW32[k] = (float)invW[k]; }
  for (int e = 0; e < 4 * nsv; ++e) dcp32[e] = (float)dcp[e];

  L.ld = (L.n % 2 == 1) ? L.n : L.n + 1;   // odd stride: column walks hit distinct banks
  L.ws_doubles = ws_offsets(L, false).total;
  L.ws_doubles32 = ws_offsets(L, true).total;
  out.swap(S.buf);
  return MRI_OK;
}

int parse_and_build(const void* blob, size_t nbytes, Layout& L, std::vector<unsigned char>& table) {
  Blob B;
  if (!read_blob(blob, nbytes, B)) return MRI_EINVAL;
  return build_table(B, L, table);
}

}  // namespace mri

extern "C" int mri_mech_load(const void* blob, size_t nbytes, mri_mech** out) {
  if (out == nullptr) return MRI_EINVAL;
  *out = nullptr;
  mri::Layout L;
  std::vector<unsigned char> table;
  int rc = mri::parse_and_build(blob, nbytes, L, table);
  if (rc != MRI_OK) return rc;
  mri::Mech* m = new (std::nothrow) mri::Mech;
  if (!m) return MRI_ECUDA;
  m->L = L;
  if (cudaGetDevice(&m->device) != cudaSuccess || cudaMalloc(&m->d_table, table.size()) != cudaSuccess) {
    delete m;
    return MRI_ECUDA;
  }
  if (cudaMalloc(&m->d_queue, sizeof(int) * (mri::kQueueSlots + mri::kGraphQueueSlots)) != cudaSuccess) {
    cudaFree(m->d_table);
    delete m;
    return MRI_ECUDA;
  }
  if (cudaMemcpy(m->d_table, table.data(), table.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(m->d_queue);
    cudaFree(m->d_table);
    delete m;
    return MRI_ECUDA;
  }
  *out = reinterpret_cast<mri_mech*>(m);
  return MRI_OK;
}

extern "C" void mri_mech_free(mri_mech* mech) {
  if (!mech) return;
  mri::Mech* m = reinterpret_cast<mri::Mech*>(mech);
  if (m->d_table) cudaFree(m->d_table);
  if (m->d_queue) cudaFree(m->d_queue);
  delete m;
}

extern "C" int mri_mech_info(const mri_mech* mech, int* n_species, int* n_reactions) {
  if (!mech) return MRI_EINVAL;
  const mri::Mech* m = reinterpret_cast<const mri::Mech*>(mech);
  if (n_species) *n_species = m->L.Ns;
  if (n_reactions) *n_reactions = m->L.R;
  return MRI_OK;
}

extern "C" int mri_probe_mech_device(mri_mech* mech, int device) {
  if (!mech) return -1;
  mri::Mech* m = reinterpret_cast<mri::Mech*>(mech);
  const int old = m->device;
  m->device = device;
  return old;
}
