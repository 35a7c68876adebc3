// Host planning (step A0) and the C-ABI entry points.
//
// Plane-wave spheres |k+G|^2/2 <= Ecut and |q+G|^2/2 <= Ecut (Sec. II C), the
// Gamma-centred q mesh of k-point differences with the folding vector G0
// (Sec. III A, q = T q_IBZ + G0 with T = identity), the e-h pair index and the
// upper (k <= k') block list of the direct term.  Keys are exact: an integer
// for fcc, a double evaluated in a fixed order for the hexagonal sheet; this
// file is compiled with -ffp-contract=off so the tables are bit-identical to
// any other IEEE evaluation of the same expressions.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace bse {

static thread_local std::string g_last_error = "";

bse_status set_error(bse_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

bse_status cuda_check(int err, const char* what) {
  if (err == cudaSuccess) return BSE_OK;
  return set_error(BSE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString((cudaError_t)err));
}

namespace {

struct Key {
  double key;
  int g1, g2, g3;
  bool operator<(const Key& o) const { return std::tie(key, g1, g2, g3) < std::tie(o.key, o.g1, o.g2, o.g3); }
};

double cell_volume(const bse_system& s) {
  if (s.lattice == BSE_LATTICE_FCC) return s.a * s.a * s.a / 4.0;
  return s.a * s.a * std::sqrt(3.0) / 2.0 * s.c;
}

void recip_basis(const bse_system& s, double b[3][3]) {
  const double t = 2.0 * kPi / s.a;
  if (s.lattice == BSE_LATTICE_FCC) {
    const double m[3][3] = {{-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) b[i][j] = t * m[i][j];
  } else {
    b[0][0] = t; b[0][1] = t / std::sqrt(3.0); b[0][2] = 0.0;
    b[1][0] = 0.0; b[1][1] = 2.0 * t / std::sqrt(3.0); b[1][2] = 0.0;
    b[2][0] = 0.0; b[2][1] = 0.0; b[2][2] = 2.0 * kPi / s.c;
  }
}

int box_bound(const bse_system& s, int j) {
  double alen = (s.lattice == BSE_LATTICE_FCC) ? s.a / std::sqrt(2.0) : (j < 2 ? s.a : s.c);
  return (int)(std::sqrt(2.0 * s.ecut) * alen / (2.0 * kPi)) + 2;
}

// Sorted sphere of mesh offset off = (i1, i2, i3): reduced G with |off/nk + G|^2/2 <= ecut.
std::vector<int32_t> sphere(const bse_system& s, const int off[3]) {
  std::vector<Key> keys;
  const int n = s.nk[0];
  const int b0 = box_bound(s, 0), b1 = box_bound(s, 1), b2 = box_bound(s, 2);
  for (int g1 = -b0; g1 <= b0; ++g1)
    for (int g2 = -b1; g2 <= b1; ++g2)
      for (int g3 = -b2; g3 <= b2; ++g3) {
        if (s.lattice == BSE_LATTICE_FCC) {
          const long long x1 = (long long)n * g1 + off[0], x2 = (long long)n * g2 + off[1],
                          x3 = (long long)n * g3 + off[2];
          const long long q = 3 * x1 * x1 + 3 * x2 * x2 + 3 * x3 * x3 - 2 * x1 * x2 - 2 * x1 * x3 - 2 * x2 * x3;
          const double t = s.a / (2.0 * kPi);
          const double rhs = 2.0 * s.ecut * (t * t) * (double)(n * n);
          if ((double)q <= rhs) keys.push_back({(double)q, g1, g2, g3});
        } else {
          const long long x1 = (long long)n * g1 + off[0], x2 = (long long)n * g2 + off[1];
          const double sa = 2.0 * kPi / s.a;
          const double uc = 2.0 * kPi / s.c;
          const double c1 = (4.0 / 3.0) * (sa * sa);
          const double c3 = uc * uc;
          const double z = (double)(n * g3);
          const double key = c1 * (double)(x1 * x1 + x1 * x2 + x2 * x2) + c3 * (z * z);
          if (key <= 2.0 * s.ecut * (double)(n * n)) keys.push_back({key, g1, g2, g3});
        }
      }
  std::sort(keys.begin(), keys.end());
  std::vector<int32_t> out;
  out.reserve(keys.size() * 3);
  for (auto& k : keys) {
    out.push_back(k.g1);
    out.push_back(k.g2);
    out.push_back(k.g3);
  }
  return out;
}

// Grid sizes must divide the 192-entry twiddle table: 2^a 3^b with a <= 6, b <= 1.
bool is_23_smooth(int n) { return n >= 2 && n <= 64 && 192 % n == 0; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bse_status build_system(const bse_system& in, SysPlan& sp, bool device) {
  bse_system s = in;
  if (s.lattice != BSE_LATTICE_FCC && s.lattice != BSE_LATTICE_HEX) return set_error(BSE_ERR_ARG, "unknown lattice");
  if (s.lattice == BSE_LATTICE_FCC && !(s.nk[0] == s.nk[1] && s.nk[1] == s.nk[2]))
    return set_error(BSE_ERR_ARG, "fcc needs nk1 = nk2 = nk3");
  if (s.lattice == BSE_LATTICE_HEX && !(s.nk[0] == s.nk[1] && s.nk[2] == 1))
    return set_error(BSE_ERR_ARG, "hex needs nk1 = nk2 and nk3 = 1");
  if (s.nk[0] < 1 || s.nv < 1 || s.nc < 1 || s.nv > 4 || s.nc > 4)
    return set_error(BSE_ERR_ARG, "need nk >= 1 and 1 <= nv, nc <= 4");
  if (!(s.ecut > 0.0) || !(s.a > 0.0) || (s.lattice == BSE_LATTICE_HEX && !(s.c > 0.0)))
    return set_error(BSE_ERR_ARG, "ecut, a (and c) must be positive");
  for (int j = 0; j < 3; ++j)
    if (!is_23_smooth(s.fft[j])) return set_error(BSE_ERR_ARG, "fft grid sizes must divide 192 (2^a 3^b, b <= 1, <= 64)");
  if (s.coulomb != BSE_COULOMB_3D && s.coulomb != BSE_COULOMB_SLAB) return set_error(BSE_ERR_ARG, "unknown coulomb");
  const double qn = std::sqrt(s.qhat[0] * s.qhat[0] + s.qhat[1] * s.qhat[1] + s.qhat[2] * s.qhat[2]);
  if (!(qn > 0.0)) return set_error(BSE_ERR_ARG, "qhat must be nonzero");
  for (int j = 0; j < 3; ++j) s.qhat[j] /= qn;
  sp.sys = s;

  const int nk1 = s.nk[0], nk2 = s.nk[1], nk3 = s.nk[2];
  const int nkpt = nk1 * nk2 * nk3;
  DevSys& d = sp.d;
  d.nkpt = nkpt;
  d.nq = nkpt;
  d.nv = s.nv;
  d.nc = s.nc;
  d.nb = s.nv + s.nc;
  d.dim = nkpt * s.nv * s.nc;
  d.n1 = s.fft[0];
  d.n2 = s.fft[1];
  d.n3 = s.fft[2];
  d.pair_variant = -1;
  d.nk1 = nk1;
  d.nk2 = nk2;
  d.nk3 = nk3;
  d.omega_cell = cell_volume(s);
  d.norm = 1.0 / (d.omega_cell * nkpt);
  d.prefactor = 8.0 * kPi * d.norm;

  auto offs = [&](int ik, int o[3]) {
    o[0] = ik / (nk2 * nk3);
    o[1] = (ik / nk3) % nk2;
    o[2] = ik % nk3;
  };
  sp.gk.resize(nkpt);
  sp.gq.resize(nkpt);
  int npw_max = 0, ng_max = 0;
  for (int j = 0; j < 3; ++j) d.fwf[j] = d.fpair[j] = 0;
  for (int ik = 0; ik < nkpt; ++ik) {
    int o[3];
    offs(ik, o);
    sp.gk[ik] = sphere(s, o);
    sp.gq[ik] = sp.gk[ik];          // the q mesh is the k mesh
    const int n = (int)sp.gk[ik].size() / 3;
    npw_max = std::max(npw_max, n);
    ng_max = std::max(ng_max, n);
    for (int t = 0; t < n; ++t)
      for (int j = 0; j < 3; ++j) {
        const int g = sp.gk[ik][3 * t + j];
        d.fwf[j] = std::max(d.fwf[j], std::abs(g));
        d.fpair[j] = std::max(d.fpair[j], std::abs(g));
        if (o[j] != 0) d.fpair[j] = std::max(d.fpair[j], std::abs(g + 1));   // G = g - G0, G0_j = -1
      }
  }
  if (npw_max < d.nb) return set_error(BSE_ERR_ARG, "fewer plane waves than bands");
  for (int j = 0; j < 3; ++j) {
    if (s.fft[j] <= 2 * d.fwf[j] + d.fpair[j])
      return set_error(BSE_ERR_ARG, "fft grid too small for alias-free pair densities (need N > 2 Fwf + Fpair)");
    if (d.fwf[j] > 120 || d.fpair[j] > 120) return set_error(BSE_ERR_ARG, "sphere too large");
  }
  d.npw_max = npw_max;
  d.ng_max = ng_max;
  d.ng0 = (int)sp.gq[0].size() / 3;

  // upper blocks grouped by q, then by ik
  sp.qblk_off.assign(nkpt + 1, 0);
  sp.qvec_off.assign(nkpt + 1, 0);
  sp.blocks.clear();
  const long long per_blk = (long long)s.nv * s.nv + (long long)s.nc * s.nc;
  for (int iq = 0; iq < nkpt; ++iq) {
    int qo[3];
    offs(iq, qo);
    long long nb = 0;
    for (int ik = 0; ik < nkpt; ++ik) {
      int ko[3], k2[3], g0[3];
      offs(ik, ko);
      for (int j = 0; j < 3; ++j) {
        const int n = s.nk[j];
        const int t = ko[j] + qo[j];
        k2[j] = t % n;
        g0[j] = 0;
        // k' - k = q + G0  with k'_j = (k_j + q_j) mod n  =>  G0_j = -1 when the sum wraps
        if (t >= n) g0[j] = -1;
      }
      const int ik2 = (k2[0] * nk2 + k2[1]) * nk3 + k2[2];
      if (ik > ik2) continue;
      sp.blocks.insert(sp.blocks.end(), {ik, ik2, iq, g0[0], g0[1], g0[2]});
      ++nb;
    }
    sp.qblk_off[iq + 1] = sp.qblk_off[iq] + nb;
    sp.qvec_off[iq + 1] = sp.qvec_off[iq] + nb * per_blk;
  }
  d.nblocks = sp.qblk_off[nkpt];

  // ---- device tables (one allocation) ----
  double b[3][3];
  recip_basis(s, b);
  std::vector<char4> h_gk((size_t)nkpt * npw_max, make_char4(0, 0, 0, 0));
  std::vector<int> h_npw(nkpt), h_ngq(nkpt);
  std::vector<double> h_kgq((size_t)nkpt * npw_max, 0.0);
  std::vector<float> h_vsq((size_t)nkpt * ng_max, 0.0f);   // sqrt(4 pi)/|q+G| on the q spheres (= k spheres)
  for (int ik = 0; ik < nkpt; ++ik) {
    int o[3];
    offs(ik, o);
    const int n = (int)sp.gk[ik].size() / 3;
    h_npw[ik] = h_ngq[ik] = n;
    for (int t = 0; t < n; ++t) {
      const int* g = &sp.gk[ik][3 * t];
      h_gk[(size_t)ik * npw_max + t] = make_char4((signed char)g[0], (signed char)g[1], (signed char)g[2], 0);
      double kg[3] = {0, 0, 0};
      for (int i = 0; i < 3; ++i) {
        const double red = (double)g[i] + (double)o[i] / (double)s.nk[i];
        for (int j = 0; j < 3; ++j) kg[j] += red * b[i][j];
      }
      h_kgq[(size_t)ik * npw_max + t] = s.qhat[0] * kg[0] + s.qhat[1] * kg[1] + s.qhat[2] * kg[2];
      const double kn = std::sqrt(kg[0] * kg[0] + kg[1] * kg[1] + kg[2] * kg[2]);
      if (kn > 0.0 && t < ng_max) h_vsq[(size_t)ik * ng_max + t] = (float)(std::sqrt(4.0 * kPi) / kn);
    }
  }
  std::vector<float> h_xs(ng_max, 0.0f);
  for (int t = 1; t < d.ng0; ++t) {
    const int* g = &sp.gq[0][3 * t];
    double p[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) p[j] += (double)g[i] * b[i][j];
    const double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    double v = 4.0 * kPi / p2;
    if (s.coulomb == BSE_COULOMB_SLAB) {
      const double zc = 0.5 * s.c;
      const double ppar = std::sqrt(p[0] * p[0] + p[1] * p[1]);
      v *= (1.0 - std::exp(-ppar * zc) * std::cos(p[2] * zc));
    }
    h_xs[t] = (float)std::sqrt(2.0 * d.norm * v);
  }

  // ---- q-point symmetry (Sec. III A) ----
  // Operations: integer matrices R on reduced reciprocal coordinates with R^T M R = M (M the
  // reciprocal metric) that map the mesh onto itself; identity first, then ascending row-major
  // entries.  Irreducible points and maps: q visited by ascending index, an unassigned q becomes
  // irreducible, each operation in order assigns its image s R q (s = +1, then -1) if unassigned,
  // with G0 = q' - s R q_IBZ.  Sphere map of q: G -> s R^-1 (G + G0) on the sphere of q_IBZ.
  {
    double M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = b[i][0] * b[j][0] + b[i][1] * b[j][1] + b[i][2] * b[j][2];
    double mmax = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) mmax = std::max(mmax, std::fabs(M[i][j]));
    std::vector<std::array<int, 9>> ops;
    std::array<int, 9> R;
    for (int code = 0; code < 19683; ++code) {
      int c = code;
      for (int t = 8; t >= 0; --t) {         // entries in -1, 0, 1, lexicographic with entry 0 most significant
        R[t] = c % 3 - 1;
        c /= 3;
      }
      const int det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                      R[2] * (R[3] * R[7] - R[4] * R[6]);
      if (det != 1 && det != -1) continue;
      bool ok = true;
      for (int i = 0; i < 3 && ok; ++i)
        for (int j = 0; j < 3 && ok; ++j) {
          double v = 0.0;                     // (R^T M R)_ij
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) v += R[3 * k + i] * M[k][l] * R[3 * l + j];
          ok = std::fabs(v - M[i][j]) <= 1e-9 * mmax;
        }
      for (int i = 0; i < 3 && ok; ++i)       // image of e_j / n_j on the mesh: R_ij n_i / n_j integral
        for (int j = 0; j < 3 && ok; ++j) ok = (R[3 * i + j] * s.nk[i]) % s.nk[j] == 0;
      if (ok) ops.push_back(R);
    }
    const std::array<int, 9> ident = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    std::vector<std::array<int, 9>> sorted;
    sorted.push_back(ident);
    for (const auto& r : ops)
      if (r != ident) sorted.push_back(r);    // enumeration order is already lexicographic
    sp.ops = sorted;
    const int nops = (int)sorted.size();
    sp.qmap.assign((size_t)6 * nkpt, -1);
    sp.ibz.clear();
    for (int iq = 0; iq < nkpt; ++iq) {
      if (sp.qmap[6 * iq] >= 0) continue;
      sp.ibz.push_back(iq);
      int o[3];
      offs(iq, o);
      for (int io = 0; io < nops; ++io)
        for (int tr = 0; tr < 2; ++tr) {
          const auto& r = sorted[io];
          int img[3], fold[3], g0[3];
          for (int i = 0; i < 3; ++i) {
            img[i] = (tr ? -1 : 1) * (r[3 * i] * o[0] + r[3 * i + 1] * o[1] + r[3 * i + 2] * o[2]);
            fold[i] = ((img[i] % s.nk[i]) + s.nk[i]) % s.nk[i];
            g0[i] = (fold[i] - img[i]) / s.nk[i];
          }
          const int iq2 = (fold[0] * nk2 + fold[1]) * nk3 + fold[2];
          if (sp.qmap[6 * iq2] >= 0) continue;
          int* m = &sp.qmap[6 * iq2];
          m[0] = (int)sp.ibz.size() - 1;
          m[1] = io;
          m[2] = tr;
          m[3] = g0[0];
          m[4] = g0[1];
          m[5] = g0[2];
        }
    }
    sp.qperm.assign((size_t)nkpt * ng_max, -1);
    auto key = [](int a, int b2, int c) { return ((long long)(a + 512) << 20) | ((long long)(b2 + 512) << 10) | (c + 512); };
    std::vector<std::unordered_map<long long, int>> pos(sp.ibz.size());
    for (size_t j = 0; j < sp.ibz.size(); ++j) {
      const auto& g = sp.gq[sp.ibz[j]];
      for (int t = 0; t < (int)g.size() / 3; ++t) pos[j][key(g[3 * t], g[3 * t + 1], g[3 * t + 2])] = t;
    }
    for (int iq = 0; iq < nkpt; ++iq) {
      const int* m = &sp.qmap[6 * iq];
      const auto& r = sorted[m[1]];
      // R^-1 = adj(R) / det(R), integral
      const int det = r[0] * (r[4] * r[8] - r[5] * r[7]) - r[1] * (r[3] * r[8] - r[5] * r[6]) +
                      r[2] * (r[3] * r[7] - r[4] * r[6]);
      int ri[9] = {(r[4] * r[8] - r[5] * r[7]) * det, (r[2] * r[7] - r[1] * r[8]) * det, (r[1] * r[5] - r[2] * r[4]) * det,
                   (r[5] * r[6] - r[3] * r[8]) * det, (r[0] * r[8] - r[2] * r[6]) * det, (r[2] * r[3] - r[0] * r[5]) * det,
                   (r[3] * r[7] - r[4] * r[6]) * det, (r[1] * r[6] - r[0] * r[7]) * det, (r[0] * r[4] - r[1] * r[3]) * det};
      const int sg = m[2] ? -1 : 1;
      const auto& g = sp.gq[iq];
      for (int t = 0; t < (int)g.size() / 3; ++t) {
        const int x[3] = {g[3 * t] + m[3], g[3 * t + 1] + m[4], g[3 * t + 2] + m[5]};
        int y[3];
        for (int i = 0; i < 3; ++i) y[i] = sg * (ri[3 * i] * x[0] + ri[3 * i + 1] * x[1] + ri[3 * i + 2] * x[2]);
        auto it = pos[m[0]].find(key(y[0], y[1], y[2]));
        if (it == pos[m[0]].end()) return set_error(BSE_ERR_ARG, "symmetry: sphere of q does not map onto its irreducible point");
        sp.qperm[(size_t)iq * ng_max + t] = it->second;
      }
    }
    d.nibz = (int)sp.ibz.size();
  }

  // ---- k-point symmetry of the blocks (Sec. III A) ----
  // With states that carry the point group, H_{Rk,Rk'} = H_{k,k'}: upper blocks visited in row-major
  // order, an unassigned block becomes a representative, and each operation in order assigns the
  // upper block of (R k, R k') to it (directly if R k <= R k', as the Hermitian mirror otherwise).
  // The plan keeps only the representatives; the others are listed for the fill stage.
  d.nfill = 0;
  sp.fill.clear();
  if (s.kpoint_symmetry) {
    const int nops = (int)sp.ops.size();
    std::vector<int> img((size_t)nops * nkpt);
    for (int io = 0; io < nops; ++io) {
      const auto& r = sp.ops[io];
      for (int ik = 0; ik < nkpt; ++ik) {
        int o[3], f[3];
        offs(ik, o);
        for (int i = 0; i < 3; ++i) {
          const int v = r[3 * i] * o[0] + r[3 * i + 1] * o[1] + r[3 * i + 2] * o[2];
          f[i] = ((v % s.nk[i]) + s.nk[i]) % s.nk[i];
        }
        img[(size_t)io * nkpt + ik] = (f[0] * nk2 + f[1]) * nk3 + f[2];
      }
    }
    auto up_index = [&](long long a, long long b2) { return a * nkpt - a * (a - 1) / 2 + (b2 - a); };
    const long long nup = (long long)nkpt * (nkpt + 1) / 2;
    std::vector<long long> rep(nup, -1);
    std::vector<char> mir(nup, 0);
    std::vector<int2> pair_of(nup);
    long long idx = 0;
    for (int a0 = 0; a0 < nkpt; ++a0)
      for (int b0 = a0; b0 < nkpt; ++b0, ++idx) {
        pair_of[idx] = make_int2(a0, b0);
        if (rep[idx] >= 0) continue;
        for (int io = 0; io < nops; ++io) {
          const int a = img[(size_t)io * nkpt + a0], b2 = img[(size_t)io * nkpt + b0];
          const long long j = a <= b2 ? up_index(a, b2) : up_index(b2, a);
          if (rep[j] < 0) {
            rep[j] = idx;
            mir[j] = a <= b2 ? 0 : 1;
          }
        }
      }
    for (long long j = 0; j < nup; ++j) {
      if (rep[j] == j) continue;
      const int2 p = pair_of[j], r = pair_of[rep[j]];
      sp.fill.push_back(make_int4(p.x, p.y, r.x, mir[j] ? -(r.y + 1) : r.y));
    }
    d.nfill = (long long)sp.fill.size();
    std::vector<int32_t> kept;
    std::vector<long long> qb(nkpt + 1, 0), qv(nkpt + 1, 0);
    const long long per_blk = (long long)s.nv * s.nv + (long long)s.nc * s.nc;
    for (int iq = 0; iq < nkpt; ++iq) {
      long long nb = 0;
      for (long long i = sp.qblk_off[iq]; i < sp.qblk_off[iq + 1]; ++i) {
        const int32_t* r = &sp.blocks[6 * i];
        if (rep[up_index(r[0], r[1])] != up_index(r[0], r[1])) continue;
        kept.insert(kept.end(), r, r + 6);
        ++nb;
      }
      qb[iq + 1] = qb[iq] + nb;
      qv[iq + 1] = qv[iq] + nb * per_blk;
    }
    sp.blocks = kept;
    sp.qblk_off = qb;
    sp.qvec_off = qv;
    d.nblocks = qb[nkpt];
  }
  std::vector<int4> h_blocks(d.nblocks > 0 ? d.nblocks : 1);
  for (long long i = 0; i < d.nblocks; ++i) {
    const int32_t* r = &sp.blocks[6 * i];
    const int packed = (r[3] + 1) | ((r[4] + 1) << 2) | ((r[5] + 1) << 4);
    h_blocks[i] = make_int4(r[0], r[1], r[2], packed);
  }
  std::vector<int> h_blkidx((size_t)nkpt * nkpt, -1);
  for (long long i = 0; i < d.nblocks; ++i) {
    const int32_t* r = &sp.blocks[6 * i];
    h_blkidx[(size_t)r[2] * nkpt + r[0]] = (int)i;
  }

  // -G on the q = 0 sphere (coupling exchange, Bx)
  std::vector<int> h_gm0(d.ng0 > 0 ? d.ng0 : 1, -1);
  {
    std::unordered_map<long long, int> pos;
    auto key = [](int a, int b2, int c) { return ((long long)(a + 512) << 20) | ((long long)(b2 + 512) << 10) | (c + 512); };
    for (int t = 0; t < d.ng0; ++t) pos[key(sp.gq[0][3 * t], sp.gq[0][3 * t + 1], sp.gq[0][3 * t + 2])] = t;
    sp.gminus0_complete = true;
    for (int t = 0; t < d.ng0; ++t) {
      auto it = pos.find(key(-sp.gq[0][3 * t], -sp.gq[0][3 * t + 1], -sp.gq[0][3 * t + 2]));
      if (it == pos.end()) sp.gminus0_complete = false;
      else h_gm0[t] = it->second;
    }
  }

  // ---- tensor-core direct densities: k' regions, their K layouts, sphere positions ----
  // Regions hold at most 96 / max(Nv, Nc) mesh points (one MMA N tile of (k', band) columns, at most 96 so
  // that two accumulators and two A tiles fit in tensor memory).  When a
  // plane of the mesh holds that many, regions are one plane thick in k'_1 (the q chunks are ranges of
  // q, i.e. slabs in q_1); the divisors of the mesh with the largest product are taken, then the most
  // compact (smallest largest extent n_j / nk_j).
  std::vector<char4> h_klist;
  std::vector<int> h_kcount;
  std::vector<short> h_kpos((size_t)nkpt * npw_max, 0), h_pmap;
  {
    const int rmax = 96 / std::max(s.nv, s.nc);
    const bool thin = nk2 * nk3 >= rmax;
    int best[3] = {1, 1, 1};
    long long best_p = 0;
    double best_e = 1e30;
    for (int r1 = 1; r1 <= nk1; ++r1)
      for (int r2 = 1; r2 <= nk2; ++r2)
        for (int r3 = 1; r3 <= nk3; ++r3) {
          if (nk1 % r1 || nk2 % r2 || nk3 % r3) continue;
          if (thin && r1 != 1) continue;
          const long long pr = (long long)r1 * r2 * r3;
          if (pr > rmax) continue;
          const double e = std::max({(double)r1 / nk1, (double)r2 / nk2, (double)r3 / nk3});
          if (pr > best_p || (pr == best_p && e < best_e - 1e-12)) {
            best_p = pr;
            best_e = e;
            best[0] = r1;
            best[1] = r2;
            best[2] = r3;
          }
        }
    for (int j = 0; j < 3; ++j) {
      d.tc_rg[j] = best[j];
      d.tc_nr[j] = s.nk[j] / best[j];
    }
    d.tc_nreg = d.tc_nr[0] * d.tc_nr[1] * d.tc_nr[2];
    d.tc_rsize = best[0] * best[1] * best[2];
    std::vector<std::vector<std::array<int, 3>>> lists(d.tc_nreg);
    for (int ik = 0; ik < nkpt; ++ik) {
      int o[3];
      offs(ik, o);
      const int r = ((o[0] / best[0]) * d.tc_nr[1] + o[1] / best[1]) * d.tc_nr[2] + o[2] / best[2];
      const auto& g = sp.gk[ik];
      for (int t = 0; t < (int)g.size() / 3; ++t) lists[r].push_back({g[3 * t], g[3 * t + 1], g[3 * t + 2]});
    }
    int kmax = 0;
    for (auto& l : lists) {
      std::sort(l.begin(), l.end());
      l.erase(std::unique(l.begin(), l.end()), l.end());
      kmax = std::max(kmax, (int)l.size());
    }
    d.tc_kpad = (kmax + 31) / 32 * 32;
    h_klist.assign((size_t)d.tc_nreg * d.tc_kpad, make_char4(0, 0, 0, 1));   // w = 1: padding
    h_kcount.assign(d.tc_nreg, 0);
    for (int r = 0; r < d.tc_nreg; ++r) {
      h_kcount[r] = (int)lists[r].size();
      for (size_t t = 0; t < lists[r].size(); ++t)
        h_klist[(size_t)r * d.tc_kpad + t] =
            make_char4((signed char)lists[r][t][0], (signed char)lists[r][t][1], (signed char)lists[r][t][2], 0);
    }
    for (int ik = 0; ik < nkpt; ++ik) {
      int o[3];
      offs(ik, o);
      const int r = ((o[0] / best[0]) * d.tc_nr[1] + o[1] / best[1]) * d.tc_nr[2] + o[2] / best[2];
      const auto& g = sp.gk[ik];
      for (int t = 0; t < (int)g.size() / 3; ++t) {
        const std::array<int, 3> key = {g[3 * t], g[3 * t + 1], g[3 * t + 2]};
        const auto it = std::lower_bound(lists[r].begin(), lists[r].end(), key);
        h_kpos[(size_t)ik * npw_max + t] = (short)(it - lists[r].begin());
      }
    }
    const int p0 = 2 * d.fwf[0] + 1, p1 = 2 * d.fwf[1] + 1, p2 = 2 * d.fwf[2] + 1;
    h_pmap.assign((size_t)nkpt * p0 * p1 * p2, (short)-1);
    for (int iq = 0; iq < nkpt; ++iq) {
      const auto& g = sp.gq[iq];
      for (int t = 0; t < (int)g.size() / 3; ++t)
        h_pmap[(size_t)iq * p0 * p1 * p2 + ((size_t)(g[3 * t] + d.fwf[0]) * p1 + g[3 * t + 1] + d.fwf[1]) * p2 +
               g[3 * t + 2] + d.fwf[2]] = (short)t;
    }
  }

  if (!device) return BSE_OK;
  size_t off = 0;
  const size_t o_gk = off; off = align256(off + h_gk.size() * sizeof(char4));
  const size_t o_npw = off; off = align256(off + h_npw.size() * sizeof(int));
  const size_t o_ngq = off; off = align256(off + h_ngq.size() * sizeof(int));
  const size_t o_blk = off; off = align256(off + h_blocks.size() * sizeof(int4));
  const size_t o_qbo = off; off = align256(off + sp.qblk_off.size() * sizeof(long long));
  const size_t o_qvo = off; off = align256(off + sp.qvec_off.size() * sizeof(long long));
  const size_t o_kgq = off; off = align256(off + h_kgq.size() * sizeof(double));
  const size_t o_xs = off; off = align256(off + h_xs.size() * sizeof(float));
  const size_t o_bi = off; off = align256(off + h_blkidx.size() * sizeof(int));
  const size_t o_vsq = off; off = align256(off + h_vsq.size() * sizeof(float));
  const size_t o_gm0 = off; off = align256(off + h_gm0.size() * sizeof(int));
  std::vector<int2> h_qsym(nkpt);
  for (int iq = 0; iq < nkpt; ++iq) h_qsym[iq] = make_int2(sp.qmap[6 * iq], sp.qmap[6 * iq + 2]);
  const size_t o_qp = off; off = align256(off + sp.qperm.size() * sizeof(int));
  const size_t o_qs = off; off = align256(off + h_qsym.size() * sizeof(int2));
  const size_t o_fill = off; off = align256(off + (sp.fill.empty() ? 1 : sp.fill.size()) * sizeof(int4));
  const size_t o_tkl = off; off = align256(off + h_klist.size() * sizeof(char4));
  const size_t o_tkc = off; off = align256(off + h_kcount.size() * sizeof(int));
  const size_t o_tkp = off; off = align256(off + h_kpos.size() * sizeof(short));
  const size_t o_tpm = off; off = align256(off + h_pmap.size() * sizeof(short));
  char* base = nullptr;
  bse_status st = cuda_check(cudaMalloc((void**)&base, off), "cudaMalloc(plan tables)");
  if (st != BSE_OK) return st;
  sp.dmem = base;
  auto up = [&](size_t o, const void* src, size_t bytes) {
    return bytes ? cudaMemcpy(base + o, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  int err = up(o_gk, h_gk.data(), h_gk.size() * sizeof(char4));
  if (!err) err = up(o_npw, h_npw.data(), h_npw.size() * sizeof(int));
  if (!err) err = up(o_ngq, h_ngq.data(), h_ngq.size() * sizeof(int));
  if (!err) err = up(o_blk, h_blocks.data(), h_blocks.size() * sizeof(int4));
  if (!err) err = up(o_qbo, sp.qblk_off.data(), sp.qblk_off.size() * sizeof(long long));
  if (!err) err = up(o_qvo, sp.qvec_off.data(), sp.qvec_off.size() * sizeof(long long));
  if (!err) err = up(o_kgq, h_kgq.data(), h_kgq.size() * sizeof(double));
  if (!err) err = up(o_xs, h_xs.data(), h_xs.size() * sizeof(float));
  if (!err) err = up(o_bi, h_blkidx.data(), h_blkidx.size() * sizeof(int));
  if (!err) err = up(o_vsq, h_vsq.data(), h_vsq.size() * sizeof(float));
  if (!err) err = up(o_gm0, h_gm0.data(), h_gm0.size() * sizeof(int));
  if (!err) err = up(o_qp, sp.qperm.data(), sp.qperm.size() * sizeof(int));
  if (!err) err = up(o_qs, h_qsym.data(), h_qsym.size() * sizeof(int2));
  if (!err) err = up(o_fill, sp.fill.data(), sp.fill.size() * sizeof(int4));
  if (!err) err = up(o_tkl, h_klist.data(), h_klist.size() * sizeof(char4));
  if (!err) err = up(o_tkc, h_kcount.data(), h_kcount.size() * sizeof(int));
  if (!err) err = up(o_tkp, h_kpos.data(), h_kpos.size() * sizeof(short));
  if (!err) err = up(o_tpm, h_pmap.data(), h_pmap.size() * sizeof(short));
  if ((st = cuda_check(err, "cudaMemcpy(plan tables)")) != BSE_OK) return st;
  d.gk = (const char4*)(base + o_gk);
  d.npw = (const int*)(base + o_npw);
  d.gq = d.gk;                        // same spheres (q mesh = k mesh)
  d.ngq = (const int*)(base + o_ngq);
  d.blocks = (const int4*)(base + o_blk);
  d.qblk_off = (const long long*)(base + o_qbo);
  d.qvec_off = (const long long*)(base + o_qvo);
  d.kgq = (const double*)(base + o_kgq);
  d.xscale = (const float*)(base + o_xs);
  d.blkidx = (const int*)(base + o_bi);
  d.vsq = (const float*)(base + o_vsq);
  d.gminus0 = (const int*)(base + o_gm0);
  d.qperm = (const int*)(base + o_qp);
  d.qsym = (const int2*)(base + o_qs);
  d.fill = (const int4*)(base + o_fill);
  d.tc_klist = (const char4*)(base + o_tkl);
  d.tc_kcount = (const int*)(base + o_tkc);
  d.tc_kpos = (const short*)(base + o_tkp);
  d.tc_pmap = (const short*)(base + o_tpm);
  return BSE_OK;
}

bse_status check_plan(const bse_plan* plan, int s) {
  if (!plan) return set_error(BSE_ERR_ARG, "plan is NULL");
  if (s < 0 || s >= (int)plan->sys.size()) return set_error(BSE_ERR_ARG, "system index out of range");
  return BSE_OK;
}

bse_status check_device_plan(const bse_plan* plan, int s) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  if (!plan->d_status) return set_error(BSE_ERR_ARG, "host-only plan: no device tables");
  return BSE_OK;
}

// Non-finite scan of one caller input (see launch_nonfinite_scan); NULL or empty inputs are skipped.
bse_status scan_input(const bse_plan* plan, const void* p, long long n, int elem_bytes, void* stream) {
  return cuda_check(launch_nonfinite_scan(p, n, elem_bytes, plan->d_status, stream), "input scan");
}

bse_status create(const bse_system* sys, int nsys, bse_plan** out, bool device) {
  if (!sys || nsys < 1 || !out) return set_error(BSE_ERR_ARG, "need sys, nsys >= 1 and out");
  *out = nullptr;
  bse_plan* p = new bse_plan();
  if (device) cudaGetDevice(&p->device);
  p->sys.resize(nsys);
  bse_status st = BSE_OK;
  for (int i = 0; i < nsys && st == BSE_OK; ++i) st = build_system(sys[i], p->sys[i], device);
  if (device) {
    if (st == BSE_OK) st = cuda_check(cudaMalloc((void**)&p->d_status, sizeof(int)), "cudaMalloc(status)");
    if (st == BSE_OK) st = cuda_check(cudaMemset(p->d_status, 0, sizeof(int)), "cudaMemset(status)");
    if (st == BSE_OK) st = cuda_check(upload_twiddles(), "twiddle upload");
  }
  if (st != BSE_OK) {
    std::string msg = g_last_error;
    bse_plan_destroy(p);
    return set_error(st, msg);
  }
  *out = p;
  return BSE_OK;
}

}  // namespace
}  // namespace bse

using namespace bse;

extern "C" {

const char* bse_last_error(void) { return g_last_error.c_str(); }

bse_status bse_plan_create(const bse_system* sys, int nsys, bse_plan** out) { return create(sys, nsys, out, true); }

bse_status bse_plan_create_host(const bse_system* sys, int nsys, bse_plan** out) {
  return create(sys, nsys, out, false);
}

bse_status bse_plan_destroy(bse_plan* plan) {
  if (!plan) return BSE_OK;
  for (auto& sp : plan->sys)
    if (sp.dmem) cudaFree(sp.dmem);
  if (plan->d_status) cudaFree(plan->d_status);
  delete plan;
  return BSE_OK;
}

bse_status bse_plan_info(const bse_plan* plan, int s, bse_info* info) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  if (!info) return set_error(BSE_ERR_ARG, "info is NULL");
  const DevSys& d = plan->sys[s].d;
  info->nkpt = d.nkpt;
  info->nb = d.nb;
  info->dim = d.dim;
  info->npw_max = d.npw_max;
  info->ng_max = d.ng_max;
  info->ng0 = d.ng0;
  info->nq = d.nq;
  info->nblocks = d.nblocks;
  info->omega_cell = d.omega_cell;
  info->norm = d.norm;
  info->prefactor = d.prefactor;
  info->kpoint_symmetry = plan->sys[s].sys.kpoint_symmetry ? 1 : 0;
  info->nfill = d.nfill;
  info->tensor_pair = tcpair_valid(d);
  for (int j = 0; j < 3; ++j) info->tc_region[j] = d.tc_rg[j];
  info->tc_kpad = d.tc_kpad;
  return BSE_OK;
}

bse_status bse_gvectors(const bse_plan* plan, int s, int kq, int is_q, int32_t* out, int* n) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  if (kq < 0 || kq >= sp.d.nkpt || !n) return set_error(BSE_ERR_ARG, "bad mesh index or n");
  const auto& v = is_q ? sp.gq[kq] : sp.gk[kq];
  *n = (int)v.size() / 3;
  if (out) std::memcpy(out, v.data(), v.size() * sizeof(int32_t));
  return BSE_OK;
}

bse_status bse_pair_blocks(const bse_plan* plan, int s, int iq, int32_t* out, int32_t* g0, int* n) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  if (iq < 0 || iq >= sp.d.nq || !n) return set_error(BSE_ERR_ARG, "bad q index or n");
  const long long b0 = sp.qblk_off[iq], b1 = sp.qblk_off[iq + 1];
  *n = (int)(b1 - b0);
  for (long long b = b0; b < b1; ++b) {
    const int32_t* r = &sp.blocks[6 * b];
    if (out) {
      out[2 * (b - b0)] = r[0];
      out[2 * (b - b0) + 1] = r[1];
    }
    if (g0)
      for (int j = 0; j < 3; ++j) g0[3 * (b - b0) + j] = r[3 + j];
  }
  return BSE_OK;
}

bse_status bse_workspace_size(const bse_plan* plan, int s, int kind, long long arg, size_t* bytes) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  if (!bytes) return set_error(BSE_ERR_ARG, "bytes is NULL");
  const DevSys& d = plan->sys[s].d;
  switch (kind) {
    case BSE_WS_PAIR:
      *bytes = pair_ws_bytes(d);
      return BSE_OK;
    case BSE_WS_KERNEL:
      if (arg < 1 || arg > d.nq) return set_error(BSE_ERR_ARG, "q chunk out of range");
      *bytes = kernel_ws_bytes(d, arg);
      return BSE_OK;
    case BSE_WS_SPECTRUM:
      if (arg < 1) return set_error(BSE_ERR_ARG, "nsteps must be >= 1");
      *bytes = spectrum_ws_bytes(d, arg);
      return BSE_OK;
    case BSE_WS_BACKWARD:
      if (arg < 1) return set_error(BSE_ERR_ARG, "nsteps must be >= 1");
      *bytes = backward_ws_bytes(d, arg);
      return BSE_OK;
    case BSE_WS_SCREEN:
      if (arg < 1 || arg > d.nq) return set_error(BSE_ERR_ARG, "q chunk out of range");
      *bytes = screen_ws_bytes(d, arg);
      return BSE_OK;
    case BSE_WS_COUPLING:
      if (arg < 0 || arg > d.nq) return set_error(BSE_ERR_ARG, "q chunk out of range");
      *bytes = coupling_ws_bytes(d, arg);
      return BSE_OK;
    case BSE_WS_COUPLED:
      if (arg < 1) return set_error(BSE_ERR_ARG, "nsteps < 1");
      *bytes = coupled_ws_bytes(d, arg);
      return BSE_OK;
    case BSE_WS_RITZ:
      if (arg < 1 || arg > 4096) return set_error(BSE_ERR_ARG, "nsteps outside [1, 4096]");
      *bytes = ritz_ws_bytes(arg);
      return BSE_OK;
    case BSE_WS_CHI0:
      *bytes = chi0_ws_bytes(d);
      return BSE_OK;
    case BSE_WS_ALDA:
      *bytes = alda_ws_bytes(d);
      return BSE_OK;
    case BSE_WS_EPSM:
      if (arg < 1) return set_error(BSE_ERR_ARG, "nw must be >= 1");
      *bytes = epsm_ws_bytes(d, arg);
      return BSE_OK;
    case BSE_WS_STATES:
      if (arg < 1 || arg > d.dim) return set_error(BSE_ERR_ARG, "n outside [1, dim]");
      *bytes = states_ws_bytes(d, arg);
      return BSE_OK;
  }
  return set_error(BSE_ERR_ARG, "unknown workspace kind");
}

bse_status bse_rho_dir_count(const bse_plan* plan, int s, int q_begin, int q_end, long long* nvec) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  if (!nvec || q_begin < 0 || q_end > sp.d.nq || q_begin > q_end) return set_error(BSE_ERR_ARG, "bad q range");
  *nvec = sp.qvec_off[q_end] - sp.qvec_off[q_begin];
  return BSE_OK;
}

bse_status bse_pair_densities(bse_plan* plan, int s, unsigned flags, const void* coef, const double* energies,
                              void* rho_x, void* P, void* rho_dir, int q_begin, int q_end, void* ws,
                              size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  const DevSys& d = sp.d;
  size_t need = 0;
  bse_workspace_size(plan, s, BSE_WS_PAIR, 0, &need);
  if (!ws || ws_bytes < need) return set_error(BSE_ERR_WORKSPACE, "pair workspace too small");
  if (!pair_supported(d)) return set_error(BSE_ERR_UNSUPPORTED, "no pair-FFT kernel compiled for this grid/sphere");
  if (flags & BSE_PD_REALSPACE) {
    if (!coef) return set_error(BSE_ERR_ARG, "coef is NULL");
    if ((st = scan_input(plan, coef, 2LL * d.nkpt * d.nb * d.npw_max, 4, stream)) != BSE_OK) return st;
    if ((st = cuda_check(launch_realspace(d, coef, ws, stream), "realspace")) != BSE_OK) return st;
  }
  if (flags & BSE_PD_EXCHANGE) {
    if (!rho_x && !P) return set_error(BSE_ERR_ARG, "exchange stage needs rho_x or P");
    if (rho_x && (st = cuda_check(launch_pair_exchange(d, ws, rho_x, plan->d_status, stream), "pair exchange")) != BSE_OK) return st;
    if (P) {
      if (!coef || !energies) return set_error(BSE_ERR_ARG, "dipole needs coef and energies");
      if ((st = scan_input(plan, energies, (long long)d.nkpt * d.nb, 8, stream)) != BSE_OK) return st;
      if ((st = cuda_check(launch_dipole(d, coef, energies, sp.sys.gap_floor, P, stream), "dipole")) != BSE_OK)
        return st;
    }
  }
  if (((flags & BSE_PD_DIRECT) != 0) + ((flags & BSE_PD_CHI0) != 0) + ((flags & BSE_PD_COUPLING) != 0) > 1)
    return set_error(BSE_ERR_ARG, "BSE_PD_DIRECT, BSE_PD_CHI0 and BSE_PD_COUPLING all write rho_dir");
  if (flags & BSE_PD_COUPLING) {
    if (!rho_dir || q_begin < 0 || q_end > d.nq || q_begin >= q_end) return set_error(BSE_ERR_ARG, "bad coupling range");
    if (sp.sys.kpoint_symmetry)
      return set_error(BSE_ERR_UNSUPPORTED, "the coupling densities are built without k-point symmetry");
    const long long vb = 2LL * d.nv * d.nc * sp.qblk_off[q_begin];
    if ((st = cuda_check(launch_pair_coupling(d, ws, rho_dir, q_begin, q_end, vb, plan->d_status, stream),
                         "pair coupling")) != BSE_OK)
      return st;
  }
  if (flags & BSE_PD_CHI0) {
    if (!rho_dir || q_begin < 0 || q_end > d.nq || q_begin >= q_end) return set_error(BSE_ERR_ARG, "bad chi0 range");
    if ((st = cuda_check(launch_pair_chi0(d, ws, rho_dir, q_begin, q_end, plan->d_status, stream), "pair chi0")) !=
        BSE_OK)
      return st;
  }
  if (flags & BSE_PD_DIRECT) {
    if (!rho_dir || q_begin < 0 || q_end > d.nq || q_begin >= q_end) return set_error(BSE_ERR_ARG, "bad direct range");
    const long long vb = sp.qvec_off[q_begin];
    if (flags & BSE_PD_TENSOR) {
      if (!tcpair_valid(d)) return set_error(BSE_ERR_UNSUPPORTED, "no tensor-core route for this system");
      if ((st = cuda_check(launch_pair_direct_tensor(d, ws, rho_dir, q_begin, q_end, vb, plan->d_status, stream),
                           "pair direct (tensor)")) != BSE_OK)
        return st;
    } else if ((st = cuda_check(launch_pair_direct(d, ws, rho_dir, q_begin, q_end, vb, plan->d_status, stream),
                                "pair direct")) != BSE_OK)
      return st;
  }
  return BSE_OK;
}

bse_status bse_pair_variants(const bse_plan* plan, int s, bse_pair_variant* out, int cap, int* count, int* current) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  if (!count || !current || cap < 0 || (cap > 0 && !out)) return set_error(BSE_ERR_ARG, "bad output arguments");
  const DevSys& d = plan->sys[s].d;
  int buf[7 * 64];
  const int n = pair_variants(d, buf, 64);
  for (int i = 0; i < n && i < cap && i < 64; ++i) {
    const int* b = buf + 7 * i;
    out[i] = bse_pair_variant{b[0], b[1], b[2], b[3], b[4], b[5], b[6]};
  }
  *count = n;
  *current = pair_variant_current(d);
  return BSE_OK;
}

bse_status bse_set_pair_variant(bse_plan* plan, int s, int index) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  DevSys& d = plan->sys[s].d;
  if (index != -1) {
    int buf[7 * 65];
    const int n = pair_variants(d, buf, 64);
    bool found = false;
    for (int i = 0; i < n && i < 64; ++i) found = found || buf[7 * i] == index;
    if (!found) return set_error(BSE_ERR_ARG, "pair variant not valid for this system");
  }
  d.pair_variant = index;
  return BSE_OK;
}

bse_status bse_autotune_pair(bse_plan* plan, int s, void* ws, size_t ws_bytes, void* rho_dir, int q_begin, int q_end,
                             int reps, float* ms, int cap, int* chosen, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  SysPlan& sp = plan->sys[s];
  DevSys& d = sp.d;
  size_t need = 0;
  bse_workspace_size(plan, s, BSE_WS_PAIR, 0, &need);
  if (!ws || ws_bytes < need) return set_error(BSE_ERR_WORKSPACE, "pair workspace too small");
  if (!rho_dir || q_begin < 0 || q_end > d.nq || q_begin >= q_end || reps < 1 || !chosen || cap < 0 ||
      (cap > 0 && !ms))
    return set_error(BSE_ERR_ARG, "bad autotune arguments");
  int buf[7 * 64];
  const int n = pair_variants(d, buf, 64);
  if (n == 0) return set_error(BSE_ERR_UNSUPPORTED, "no pair-FFT kernel compiled for this grid/sphere");
  cudaStream_t stm = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if ((st = cuda_check(cudaEventCreate(&e0), "event")) != BSE_OK) return st;
  if ((st = cuda_check(cudaEventCreate(&e1), "event")) != BSE_OK) {
    cudaEventDestroy(e0);
    return st;
  }
  const int saved = d.pair_variant;
  const long long vb = sp.qvec_off[q_begin];
  float best = 0.f;
  int besti = -1;
  for (int i = 0; i < n && i < 64 && st == BSE_OK; ++i) {
    d.pair_variant = buf[7 * i];
    st = cuda_check(launch_pair_direct(d, ws, rho_dir, q_begin, q_end, vb, plan->d_status, stream), "autotune warm-up");
    if (st != BSE_OK) break;
    cudaEventRecord(e0, stm);
    for (int r = 0; r < reps && st == BSE_OK; ++r)
      st = cuda_check(launch_pair_direct(d, ws, rho_dir, q_begin, q_end, vb, plan->d_status, stream), "autotune");
    cudaEventRecord(e1, stm);
    if (st == BSE_OK) st = cuda_check(cudaEventSynchronize(e1), "autotune sync");
    float t = 0.f;
    if (st == BSE_OK) st = cuda_check(cudaEventElapsedTime(&t, e0, e1), "autotune timing");
    t /= (float)reps;
    if (i < cap) ms[i] = t;
    if (st == BSE_OK && (besti < 0 || t < best)) {
      best = t;
      besti = buf[7 * i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  d.pair_variant = (st == BSE_OK) ? besti : saved;
  *chosen = d.pair_variant;
  return st;
}

bse_status bse_build_kernel(bse_plan* plan, int s, unsigned flags, const void* rho_x, const void* rho_dir,
                            int q_begin, int q_end, const void* W, const double* energies, double delta, int prec,
                            void* H, void* ws, size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!H) return set_error(BSE_ERR_ARG, "H is NULL");
  if (prec != BSE_PREC_FP32 && prec != BSE_PREC_BF16X3) return set_error(BSE_ERR_ARG, "unknown precision");
  if (flags & BSE_BK_INIT) {
    if (!rho_x || !energies) return set_error(BSE_ERR_ARG, "init needs rho_x and energies");
    if ((st = scan_input(plan, energies, (long long)d.nkpt * d.nb, 8, stream)) != BSE_OK) return st;
    if (prec == BSE_PREC_BF16X3 && ws) {          // the tensor-core Gram product, split images in ws
      if (ws_bytes < gram_ws_bytes(d)) return set_error(BSE_ERR_WORKSPACE, "kernel workspace too small for init");
      if ((st = cuda_check(launch_kernel_init_tc(d, rho_x, energies, delta, H, ws, plan->d_status, stream),
                           "kernel init (tensor)")) != BSE_OK)
        return st;
    } else if ((st = cuda_check(launch_kernel_init(d, rho_x, energies, delta, H, stream), "kernel init")) != BSE_OK)
      return st;
  }
  if (flags & BSE_BK_DIRECT) {
    if (!rho_dir || !W || q_begin < 0 || q_end > d.nq || q_begin >= q_end)
      return set_error(BSE_ERR_ARG, "direct stage needs rho_dir, W and a q range");
    if (!ws || ws_bytes < kernel_ws_bytes(d, q_end - q_begin))
      return set_error(BSE_ERR_WORKSPACE, "kernel workspace too small");
    const SysPlan& sp = plan->sys[s];
    const long long ng2 = (long long)d.ng_max * d.ng_max;
    if ((st = scan_input(plan, (const char*)W + (size_t)q_begin * ng2 * 8, 2 * (q_end - q_begin) * ng2, 4, stream)) !=
        BSE_OK)
      return st;
    const long long b0 = sp.qblk_off[q_begin], nb = sp.qblk_off[q_end] - b0, vb = sp.qvec_off[q_begin];
    const long long w = (d.nc * d.nc < d.nv * d.nv) ? d.nc * d.nc : d.nv * d.nv;
    long long max_rows = 0;
    for (int q = q_begin; q < q_end; ++q) max_rows = std::max(max_rows, (sp.qblk_off[q + 1] - sp.qblk_off[q]) * w);
    const int e = launch_kernel_direct_range(d, rho_dir, q_begin, q_end, b0, nb, vb, max_rows, W, prec, H, ws,
                                             plan->d_status, stream);
    if (e == -1) return set_error(BSE_ERR_UNSUPPORTED, "precision not available in this build");
    if ((st = cuda_check(e, "kernel direct")) != BSE_OK) return st;
  }
  if (flags & BSE_BK_MIRROR) {
    if (flags & BSE_BK_DIRECT) return set_error(BSE_ERR_ARG, "the direct stage already mirrors its blocks");
    if ((st = cuda_check(launch_mirror(d, H, stream), "kernel mirror")) != BSE_OK) return st;
  }
  if (flags & BSE_BK_SYMFILL) {
    if (!plan->sys[s].sys.kpoint_symmetry) return set_error(BSE_ERR_ARG, "BSE_BK_SYMFILL needs a plan with k-point symmetry");
    if ((st = cuda_check(launch_symfill(d, H, stream), "symmetry fill")) != BSE_OK) return st;
  }
  return BSE_OK;
}

bse_status bse_apply_H(bse_plan* plan, int s, const void* H, const void* X, void* Y, int nvec, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  if (!H || !X || !Y || nvec < 1) return set_error(BSE_ERR_ARG, "apply_H needs H, X, Y and nvec >= 1");
  const DevSys& dd = plan->sys[s].d;
  if ((st = scan_input(plan, H, 2LL * dd.dim * dd.dim, 4, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, X, 2LL * nvec * dd.dim, 8, stream)) != BSE_OK) return st;
  return cuda_check(launch_apply_h(plan->sys[s].d, H, X, Y, nvec, stream), "apply_H");
}

bse_status bse_spectrum(bse_plan* plan, int s, const void* H, const void* P, int nsteps, const double* omega, int nw,
                        double eta, double* eps2, double* ab, int* steps_done, void* ws, size_t ws_bytes,
                        void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!H || !P || !omega || !eps2 || !ab || !steps_done || nsteps < 1 || nw < 0 || !(eta > 0.0))
    return set_error(BSE_ERR_ARG, "spectrum needs H, P, omega, eps2, ab, steps_done, nsteps >= 1, eta > 0");
  if (nsteps > d.dim) return set_error(BSE_ERR_ARG, "nsteps > dim");
  if (!ws || ws_bytes < spectrum_ws_bytes(d, nsteps)) return set_error(BSE_ERR_WORKSPACE, "spectrum workspace too small");
  if ((st = scan_input(plan, H, 2LL * d.dim * d.dim, 4, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, P, 2LL * d.dim, 8, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, omega, nw, 8, stream)) != BSE_OK) return st;
  const int e = launch_spectrum(d, H, P, nsteps, omega, nw, eta, eps2, ab, steps_done, ws, plan->d_status, stream);
  if (e == -1) return set_error(BSE_ERR_UNSUPPORTED, "cooperative launch not possible on this device");
  return cuda_check(e, "spectrum");
}

bse_status bse_spectrum_batch(bse_plan* plan, int n, const int* systems, const void* const* H,
                              const void* const* P, int nsteps, const double* omega, int nw, double eta,
                              double* const* eps2, double* const* ab, int* const* steps_done, void* const* ws,
                              const size_t* ws_bytes, void* stream) {
  if (!plan || !plan->d_status) return set_error(BSE_ERR_ARG, "plan is NULL or host-only");
  if (n < 1 || n > 24 || !systems || !H || !P || !eps2 || !ab || !steps_done || !ws || !ws_bytes || !omega ||
      nsteps < 1 || nw < 0 || !(eta > 0.0))
    return set_error(BSE_ERR_ARG, "batch needs 1..24 systems, all per-system arrays, nsteps >= 1, eta > 0");
  std::vector<HayJob> jobs(n);
  for (int i = 0; i < n; ++i) {
    const int s = systems[i];
    bse_status st = check_device_plan(plan, s);
    if (st != BSE_OK) return st;
    const DevSys& d = plan->sys[s].d;
    if (!H[i] || !P[i] || !eps2[i] || !ab[i] || !steps_done[i] || !ws[i])
      return set_error(BSE_ERR_ARG, "NULL pointer in a batch entry");
    if (nsteps > d.dim) return set_error(BSE_ERR_ARG, "nsteps > dim of a batched system");
    if (ws_bytes[i] < spectrum_ws_bytes(d, nsteps)) return set_error(BSE_ERR_WORKSPACE, "batch workspace too small");
    jobs[i] = HayJob{&d, H[i], P[i], eps2[i], ab[i], steps_done[i], ws[i]};
  }
  for (int i = 0; i < n; ++i) {
    const DevSys& d = plan->sys[systems[i]].d;
    bse_status st = scan_input(plan, H[i], 2LL * d.dim * d.dim, 4, stream);
    if (st == BSE_OK) st = scan_input(plan, P[i], 2LL * d.dim, 8, stream);
    if (st != BSE_OK) return st;
  }
  {
    bse_status st = scan_input(plan, omega, nw, 8, stream);
    if (st != BSE_OK) return st;
  }
  const int e = run_haydock_batch(jobs.data(), n, nsteps, omega, nw, eta, plan->d_status, stream);
  if (e == -1) return set_error(BSE_ERR_UNSUPPORTED, "cooperative launch not possible on this device");
  if (e == -2) return set_error(BSE_ERR_ARG, "more batched systems than SMs");
  return cuda_check(e, "spectrum batch");
}

bse_status bse_spectrum_static(bse_plan* plan, int s, const void* H, const void* P, int nsteps, const double* omega,
                               int nw, double eta, double* eps2, double* ab, int* steps_done, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!H || !P || !omega || !eps2 || !ab || !steps_done || nsteps < 1 || nw < 0 || !(eta > 0.0))
    return set_error(BSE_ERR_ARG, "spectrum needs H, P, omega, eps2, ab, steps_done, nsteps >= 1, eta > 0");
  if (nsteps > d.dim) return set_error(BSE_ERR_ARG, "nsteps > dim");
  const size_t need = spectrum_ws_bytes(d, nsteps);
  if (need > spectrum_static_capacity())
    return set_error(BSE_ERR_ARG, "scratch of " + std::to_string(need) + " bytes exceeds the library's static " +
                                      std::to_string(spectrum_static_capacity()) +
                                      "-byte spectrum scratch; use bse_spectrum with a caller workspace");
  if ((st = scan_input(plan, H, 2LL * d.dim * d.dim, 4, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, P, 2LL * d.dim, 8, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, omega, nw, 8, stream)) != BSE_OK) return st;
  const int e = launch_spectrum_static(d, H, P, nsteps, omega, nw, eta, eps2, ab, steps_done, plan->d_status, stream);
  if (e == -1) return set_error(BSE_ERR_UNSUPPORTED, "cooperative launch not possible on this device");
  return cuda_check(e, "spectrum (static scratch)");
}

bse_status bse_spectrum_backward(bse_plan* plan, int s, const void* H, const void* P, int nsteps,
                                 const double* omega, int nw, double eta, const double* dL_deps2,
                                 const void* rho_x, const void* rho_dir, const void* W, double* dL_ddelta,
                                 void* dL_dH, void* dL_drho_x, void* dL_drho_dir, void* dL_dW, void* ws,
                                 size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!H || !P || !omega || !dL_deps2 || !dL_ddelta || nsteps < 1 || nw < 1 || !(eta > 0.0))
    return set_error(BSE_ERR_ARG, "backward needs H, P, omega, dL_deps2, dL_ddelta, nsteps >= 1, eta > 0");
  if (nsteps > d.dim) return set_error(BSE_ERR_ARG, "nsteps > dim");
  if ((dL_drho_x && !rho_x) || ((dL_drho_dir || dL_dW) && (!rho_dir || !W)))
    return set_error(BSE_ERR_ARG, "chained gradients need their forward inputs");
  if (plan->sys[s].sys.kpoint_symmetry && (dL_drho_dir || dL_dW))
    return set_error(BSE_ERR_UNSUPPORTED, "the adjoint chain through the direct term needs every block (k-point symmetry plan)");
  if (!ws || ws_bytes < backward_ws_bytes(d, nsteps)) return set_error(BSE_ERR_WORKSPACE, "backward workspace too small");
  if ((st = scan_input(plan, H, 2LL * d.dim * d.dim, 4, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, P, 2LL * d.dim, 8, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, omega, nw, 8, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, dL_deps2, nw, 8, stream)) != BSE_OK) return st;
  if (W && (st = scan_input(plan, W, 2LL * d.nq * d.ng_max * d.ng_max, 4, stream)) != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  const int e = launch_backward(d, sp.qblk_off.data(), sp.qvec_off.data(), H, P, nsteps, omega, nw, eta, dL_deps2,
                                rho_x, rho_dir, W, dL_ddelta, dL_dH, dL_drho_x, dL_drho_dir, dL_dW, ws,
                                plan->d_status, stream);
  if (e == -1) return set_error(BSE_ERR_UNSUPPORTED, "cooperative launch not possible on this device");
  return cuda_check(e, "spectrum backward");
}

bse_status bse_screening(bse_plan* plan, int s, void* rho_chi, const double* energies, const void* P, int q_begin,
                         int q_end, int iterations, void* W, float* residual, void* ws, size_t ws_bytes,
                         void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  const DevSys& d = sp.d;
  if (sp.sys.coulomb != BSE_COULOMB_3D) return set_error(BSE_ERR_UNSUPPORTED, "screening is built for bulk systems");
  if (!rho_chi || !energies || !W || q_begin < 0 || q_end > d.nq || q_begin >= q_end || iterations < 0 ||
      iterations > 64)
    return set_error(BSE_ERR_ARG, "bad screening arguments");
  if (q_begin == 0 && !P) return set_error(BSE_ERR_ARG, "q = 0 needs the dipole P");
  if (!ws || ws_bytes < screen_ws_bytes(d, q_end - q_begin)) return set_error(BSE_ERR_WORKSPACE, "workspace too small");
  if ((st = scan_input(plan, energies, (long long)d.nkpt * d.nb, 8, stream)) != BSE_OK) return st;
  if (q_begin == 0 && (st = scan_input(plan, P, 2LL * d.dim, 8, stream)) != BSE_OK) return st;
  return cuda_check(launch_screening(d, rho_chi, energies, P, q_begin, q_end, iterations, W, residual, ws,
                                     sp.sys.gap_floor, stream),
                    "screening");
}

bse_status bse_rho_cpl_count(const bse_plan* plan, int s, int q_begin, int q_end, long long* nvec) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  if (!nvec || q_begin < 0 || q_end > sp.d.nq || q_begin > q_end) return set_error(BSE_ERR_ARG, "bad q range");
  *nvec = 2LL * sp.d.nv * sp.d.nc * (sp.qblk_off[q_end] - sp.qblk_off[q_begin]);
  return BSE_OK;
}

bse_status bse_build_coupling(bse_plan* plan, int s, unsigned flags, const void* rho_x, const void* rho_cpl,
                              int q_begin, int q_end, const void* W, int prec, void* Bm, void* ws, size_t ws_bytes,
                              void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  const DevSys& d = sp.d;
  if (!Bm) return set_error(BSE_ERR_ARG, "Bm is NULL");
  if (prec != BSE_PREC_FP32 && prec != BSE_PREC_BF16X3) return set_error(BSE_ERR_ARG, "unknown precision");
  if (d.nv * d.nc > 16) return set_error(BSE_ERR_UNSUPPORTED, "coupling blocks are built for Nv Nc <= 16");
  if (sp.sys.kpoint_symmetry && (flags & BSE_BC_DIRECT))
    return set_error(BSE_ERR_UNSUPPORTED, "the coupling block is built without k-point symmetry");
  if ((flags & BSE_BC_DIRECT) && (flags & BSE_BC_MIRROR))
    return set_error(BSE_ERR_ARG, "the direct stage already mirrors its blocks");
  if (flags & BSE_BC_INIT) {
    if (!rho_x) return set_error(BSE_ERR_ARG, "init needs rho_x");
    if (!sp.gminus0_complete) return set_error(BSE_ERR_UNSUPPORTED, "q = 0 sphere is not symmetric under G -> -G");
    if (!ws || ws_bytes < coupling_ws_bytes(d, 0)) return set_error(BSE_ERR_WORKSPACE, "coupling workspace too small");
    if ((st = cuda_check(launch_coupling_init(d, rho_x, Bm, ws, stream), "coupling init")) != BSE_OK) return st;
  }
  if (flags & BSE_BC_DIRECT) {
    if (!rho_cpl || !W || q_begin < 0 || q_end > d.nq || q_begin >= q_end)
      return set_error(BSE_ERR_ARG, "direct stage needs rho_cpl, W and a q range");
    if (!ws || ws_bytes < coupling_ws_bytes(d, q_end - q_begin))
      return set_error(BSE_ERR_WORKSPACE, "coupling workspace too small");
    const long long ng2 = (long long)d.ng_max * d.ng_max;
    if ((st = scan_input(plan, (const char*)W + (size_t)q_begin * ng2 * 8, 2 * (q_end - q_begin) * ng2, 4, stream)) !=
        BSE_OK)
      return st;
    const long long w = (long long)d.nv * d.nc;
    const long long nb = sp.qblk_off[q_end] - sp.qblk_off[q_begin], vb = 2 * w * sp.qblk_off[q_begin];
    long long max_rows = 0;
    for (int q = q_begin; q < q_end; ++q) max_rows = std::max(max_rows, (sp.qblk_off[q + 1] - sp.qblk_off[q]) * w);
    const int e = launch_coupling_direct_range(d, rho_cpl, q_begin, q_end, nb, vb, max_rows, W, prec, Bm, ws,
                                               plan->d_status, stream);
    if (e == -1) return set_error(BSE_ERR_UNSUPPORTED, "precision not available in this build");
    if ((st = cuda_check(e, "coupling direct")) != BSE_OK) return st;
  }
  if (flags & BSE_BC_MIRROR) {
    if ((st = cuda_check(launch_coupling_mirror(d, Bm, stream), "coupling mirror")) != BSE_OK) return st;
  }
  return BSE_OK;
}

bse_status bse_spectrum_coupled(bse_plan* plan, int s, const void* A, const void* Bm, const void* P, int nsteps,
                                const double* omega, int nw, double eta, double* eps2, double* b, int* steps_done,
                                void* ws, size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!A || !Bm || !P || !omega || !eps2 || !b || !steps_done || nsteps < 1 || nw < 0 || !(eta > 0.0))
    return set_error(BSE_ERR_ARG, "coupled spectrum needs A, Bm, P, omega, eps2, b, steps_done, nsteps >= 1, eta > 0");
  if (nsteps > 2 * d.dim) return set_error(BSE_ERR_ARG, "nsteps > 2 dim");
  if (!ws || ws_bytes < coupled_ws_bytes(d, nsteps)) return set_error(BSE_ERR_WORKSPACE, "coupled workspace too small");
  if ((st = scan_input(plan, A, 2LL * d.dim * d.dim, 4, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, Bm, 2LL * d.dim * d.dim, 4, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, P, 2LL * d.dim, 8, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, omega, nw, 8, stream)) != BSE_OK) return st;
  const int e = launch_spectrum_coupled(d, A, Bm, P, nsteps, omega, nw, eta, eps2, b, steps_done, ws, plan->d_status,
                                        stream);
  if (e == -2) return set_error(BSE_ERR_UNSUPPORTED, "coupled spectrum is built for dim <= 65536");
  return cuda_check(e, "coupled spectrum");
}

bse_status bse_chi0_optical(bse_plan* plan, int s, const void* rho_x, const void* P, const double* energies,
                            double delta, const double* omega, int nw, double eta, void* chi0, void* ws,
                            size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  const DevSys& d = sp.d;
  if (sp.sys.coulomb != BSE_COULOMB_3D) return set_error(BSE_ERR_UNSUPPORTED, "the optical response is built for bulk systems");
  if (!sp.gminus0_complete) return set_error(BSE_ERR_UNSUPPORTED, "q = 0 sphere is not symmetric under G -> -G");
  if (!rho_x || !P || !energies || !omega || !chi0 || nw < 1 || !(eta > 0.0))
    return set_error(BSE_ERR_ARG, "chi0 needs rho_x, P, energies, omega, chi0, nw >= 1 and eta > 0");
  if (!ws || ws_bytes < chi0_ws_bytes(d)) return set_error(BSE_ERR_WORKSPACE, "chi0 workspace too small");
  if ((st = scan_input(plan, P, 2LL * d.dim, 8, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, energies, (long long)d.nkpt * d.nb, 8, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, omega, nw, 8, stream)) != BSE_OK) return st;
  return cuda_check(launch_chi0_optical(d, rho_x, P, energies, delta, omega, nw, eta, chi0, ws, stream), "chi0");
}

bse_status bse_xc_kernel_alda(bse_plan* plan, int s, const void* pair_ws, size_t pair_bytes, void* F, void* ws,
                              size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  const DevSys& d = sp.d;
  if (sp.sys.coulomb != BSE_COULOMB_3D) return set_error(BSE_ERR_UNSUPPORTED, "the ALDA kernel is built for bulk systems");
  if (!pair_ws || !F) return set_error(BSE_ERR_ARG, "ALDA needs the pair workspace and F");
  if (pair_bytes < pair_ws_bytes(d)) return set_error(BSE_ERR_WORKSPACE, "pair workspace too small");
  if (!ws || ws_bytes < alda_ws_bytes(d)) return set_error(BSE_ERR_WORKSPACE, "ALDA workspace too small");
  int m[3] = {0, 0, 0};
  const std::vector<int32_t>& g0 = sp.gq[0];
  for (size_t t = 0; t + 2 < g0.size(); t += 3)
    for (int i = 0; i < 3; ++i) m[i] = std::max(m[i], 2 * std::abs(g0[t + i]));
  const int n[3] = {d.n1, d.n2, d.n3};
  for (int i = 0; i < 3; ++i)
    if (2 * m[i] + 1 > n[i]) return set_error(BSE_ERR_UNSUPPORTED, "grid too small for the G - G' box of the q = 0 sphere");
  return cuda_check(launch_alda_kernel(d, pair_ws, m, F, ws, stream), "ALDA kernel");
}

bse_status bse_epsilon_macro(bse_plan* plan, int s, const void* chi0, const void* F, int nw, void* eps_m, void* ws,
                             size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!chi0 || !eps_m || nw < 1) return set_error(BSE_ERR_ARG, "eps_M needs chi0, eps_m and nw >= 1");
  if (d.ng0 > 4096) return set_error(BSE_ERR_UNSUPPORTED, "q = 0 sphere larger than 4096");
  if (!ws || ws_bytes < epsm_ws_bytes(d, nw)) return set_error(BSE_ERR_WORKSPACE, "eps_M workspace too small");
  if ((st = scan_input(plan, chi0, 2LL * nw * d.ng0 * d.ng0, 4, stream)) != BSE_OK) return st;
  if (F && (st = scan_input(plan, F, 2LL * d.ng0 * d.ng0, 4, stream)) != BSE_OK) return st;
  return cuda_check(launch_epsilon_macro(d, chi0, F, nw, eps_m, ws, stream), "eps_M");
}

bse_status bse_exciton_states(bse_plan* plan, int s, const void* H, const void* X0, int n, double* theta, void* A,
                              double* ab, int* steps_done, void* ws, size_t ws_bytes, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!H || !X0 || !theta || !ab || !steps_done || n < 1 || n > d.dim)
    return set_error(BSE_ERR_ARG, "exciton states need H, X0, theta, ab, steps_done and 1 <= n <= dim");
  if (!ws || ws_bytes < states_ws_bytes(d, n)) return set_error(BSE_ERR_WORKSPACE, "exciton-state workspace too small");
  if ((st = scan_input(plan, H, 2LL * d.dim * d.dim, 4, stream)) != BSE_OK) return st;
  if ((st = scan_input(plan, X0, 2LL * d.dim, 8, stream)) != BSE_OK) return st;
  const int e = launch_exciton_states(d, H, X0, n, theta, A, ab, steps_done, ws, plan->d_status, stream);
  if (e == -1) return set_error(BSE_ERR_UNSUPPORTED, "cooperative launch not possible on this device");
  return cuda_check(e, "exciton states");
}

bse_status bse_symmetry(const bse_plan* plan, int s, int* nops, int* nibz, int32_t* ibz, int32_t* qmap,
                        int32_t* perm) {
  bse_status st = check_plan(plan, s);
  if (st != BSE_OK) return st;
  const SysPlan& sp = plan->sys[s];
  if (nops) *nops = (int)sp.ops.size();
  if (nibz) *nibz = (int)sp.ibz.size();
  if (ibz) std::memcpy(ibz, sp.ibz.data(), sp.ibz.size() * sizeof(int32_t));
  if (qmap) std::memcpy(qmap, sp.qmap.data(), sp.qmap.size() * sizeof(int32_t));
  if (perm) std::memcpy(perm, sp.qperm.data(), sp.qperm.size() * sizeof(int32_t));
  return BSE_OK;
}

bse_status bse_unfold_w(bse_plan* plan, int s, const void* W_ibz, void* W, int q_begin, int q_end, void* stream) {
  bse_status st = check_device_plan(plan, s);
  if (st != BSE_OK) return st;
  const DevSys& d = plan->sys[s].d;
  if (!W_ibz || !W || q_begin < 0 || q_end > d.nq || q_begin >= q_end) return set_error(BSE_ERR_ARG, "bad unfold arguments");
  if ((st = scan_input(plan, W_ibz, 2LL * d.nibz * d.ng_max * d.ng_max, 4, stream)) != BSE_OK) return st;
  return cuda_check(launch_unfold_w(d, W_ibz, W, q_begin, q_end, stream), "unfold W");
}

bse_status bse_ritz(const double* ab, const int* steps_done, int nsteps, double* theta, double* weight, void* ws,
                    size_t ws_bytes, void* stream) {
  if (!ab || !steps_done || !theta || !weight || nsteps < 1 || nsteps > 4096)
    return set_error(BSE_ERR_ARG, "ritz needs ab, steps_done, theta, weight and 1 <= nsteps <= 4096");
  if (!ws || ws_bytes < ritz_ws_bytes(nsteps)) return set_error(BSE_ERR_WORKSPACE, "ritz workspace too small");
  return cuda_check(launch_ritz(ab, steps_done, nsteps, theta, weight, ws, stream), "ritz");
}

bse_status bse_set_wait_limit(unsigned long long ns) {
  return cuda_check(set_wait_limit(ns), "set wait limit");
}

bse_status bse_status_read(bse_plan* plan, void* stream) {
  if (!plan || !plan->d_status) return set_error(BSE_ERR_ARG, "plan is NULL or host-only");
  bse_status st = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
  if (st != BSE_OK) return st;
  int h = 0;
  if ((st = cuda_check(cudaMemcpy(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read")) != BSE_OK)
    return st;
  cudaMemset(plan->d_status, 0, sizeof(int));
  if (h != 0) return set_error((bse_status)h, "device-side status set by a kernel");
  return BSE_OK;
}

}  // extern "C"
