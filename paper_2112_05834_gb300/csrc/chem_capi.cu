// Host side of the C ABI declared in include/chem.h: mechanism validation and
// device-table construction, handle options, launch configuration, per-cell
// statistics and the diagnostic entry points.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "chem.h"
#include "chem_capi_internal.h"
#include "chem_internal.h"
#include "chem_kernels.h"
#include "chem_mlp_internal.h"
#include "rodas4.h"
#include "ros34pw2.h"

using namespace chem;

static thread_local std::string g_create_error;

static std::string cuda_msg(const char* what, cudaError_t e) {
  return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

#define CHEM_CUDA(h, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) {                                 \
      (h)->err = cuda_msg(#call, e_);                        \
      return e_ == cudaErrorMemoryAllocation ? CHEM_ERR_OOM : CHEM_ERR_CUDA; \
    }                                                        \
  } while (0)

// ---------------------------------------------------------------------------
// Rosenbrock methods in the device stepper's transformed form
// ---------------------------------------------------------------------------
// RODAS4 is published in that form (rodas4.h). ROS34PW2 is published in the
// original form (ros34pw2.h) and converted with u_i = sum_j gamma_ij k_j
// (Hairer & Wanner II, Sec. IV.7): a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1,
// m = b^T Gamma^-1, e = (b - bhat)^T Gamma^-1.
MethodTab chem::method_tableau(int method) {
  MethodTab t{};
  if (method == METHOD_ROS34PW2) {
    const int S = 4;
    t.s = S;
    t.q = 3;
    t.e_last = 0;
    t.gamma = kRos34Gamma;
    double G[4][4] = {}, Gi[4][4] = {};
    for (int i = 0; i < S; ++i)
      for (int j = 0; j < S; ++j) G[i][j] = i == j ? kRos34Gamma : kRos34Gam[i][j];
    // inverse of the lower triangular Gamma, column by column (forward substitution)
    for (int j = 0; j < S; ++j)
      for (int i = j; i < S; ++i) {
        double v = i == j ? 1.0 : 0.0;
        for (int l = j; l < i; ++l) v -= G[i][l] * Gi[l][j];
        Gi[i][j] = v / G[i][i];
      }
    for (int i = 0; i < S; ++i)
      for (int j = 0; j < S; ++j) {
        double a = 0.0;
        for (int l = 0; l < S; ++l) a += kRos34Alpha[i][l] * Gi[l][j];
        t.a[i][j] = j < i ? a : 0.0;
        t.c[i][j] = j < i ? -Gi[i][j] : 0.0;  // the diagonal 1/gamma - Gi_ii is zero
      }
    for (int j = 0; j < S; ++j) {
      double m = 0.0, e = 0.0;
      for (int l = 0; l < S; ++l) {
        m += kRos34B[l] * Gi[l][j];
        e += (kRos34B[l] - kRos34Bhat[l]) * Gi[l][j];
      }
      t.m[j] = m;
      t.e[j] = e;
    }
    return t;
  }
  t.s = 6;
  t.q = 4;
  t.e_last = 1;
  t.gamma = kRodasGamma;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) {
      t.a[i][j] = kRodasA[i][j];
      t.c[i][j] = kRodasC[i][j];
    }
    t.m[i] = kRodasM[i];
    t.e[i] = kRodasE[i];
  }
  return t;
}

// ---------------------------------------------------------------------------
// mechanism validation
// ---------------------------------------------------------------------------
static double h_RT(const double* a, double T) {
  return a[0] + a[1] * T / 2 + a[2] * T * T / 3 + a[3] * T * T * T / 4 + a[4] * T * T * T * T / 5 + a[5] / T;
}
static double s_R(const double* a, double T) {
  return a[0] * std::log(T) + a[1] * T + a[2] * T * T / 2 + a[3] * T * T * T / 3 + a[4] * T * T * T * T / 4 + a[6];
}

static std::string validate(const chem_mechanism_desc* d) {
  const int K = d->n_species, I = d->n_reactions, E = d->n_elements;
  char buf[256];
  if (K < 1 || K > 255) return "n_species must be in [1, 255]";
  if (I < 0) return "n_reactions must be >= 0";
  if (E < 0) return "n_elements must be >= 0";
  if (!d->W || !d->nasa_lo || !d->nasa_hi || !d->T_lo || !d->T_mid || !d->T_hi)
    return "NULL species table";
  if (E > 0 && !d->elem) return "NULL element table";
  if (I > 0 && (!d->rxn_type || !d->reac_idx || !d->reac_nu || !d->prod_idx || !d->prod_nu ||
                !d->reversible || !d->A || !d->b || !d->Ea_R || !d->A0 || !d->b0 || !d->Ea0_R ||
                !d->troe || !d->eff))
    return "NULL reaction table";
  for (int k = 0; k < K; ++k) {
    if (!(d->W[k] > 0.0) || !std::isfinite(d->W[k])) {
      snprintf(buf, sizeof buf, "species %d: molecular weight must be positive", k);
      return buf;
    }
    if (!(d->T_lo[k] < d->T_mid[k] && d->T_mid[k] < d->T_hi[k])) {
      snprintf(buf, sizeof buf, "species %d: need T_lo < T_mid < T_hi", k);
      return buf;
    }
    for (int a = 0; a < 7; ++a)
      if (!std::isfinite(d->nasa_lo[7 * k + a]) || !std::isfinite(d->nasa_hi[7 * k + a])) {
        snprintf(buf, sizeof buf, "species %d: non-finite NASA coefficient", k);
        return buf;
      }
    const double Tm = d->T_mid[k];
    const double hl = h_RT(d->nasa_lo + 7 * k, Tm), hh = h_RT(d->nasa_hi + 7 * k, Tm);
    const double sl = s_R(d->nasa_lo + 7 * k, Tm), sh = s_R(d->nasa_hi + 7 * k, Tm);
    if (std::fabs(hl - hh) > 1e-6 * std::max(1.0, std::fabs(hl)) ||
        std::fabs(sl - sh) > 1e-6 * std::max(1.0, std::fabs(sl))) {
      snprintf(buf, sizeof buf, "species %d: H/RT or S/R discontinuous at T_mid", k);
      return buf;
    }
  }
  for (int i = 0; i < I; ++i) {
    const int t = d->rxn_type[i];
    if (t < 0 || t > 3) {
      snprintf(buf, sizeof buf, "reaction %d: unknown type %d", i, t);
      return buf;
    }
    for (int side = 0; side < 2; ++side) {
      const int32_t* idx = side ? d->prod_idx : d->reac_idx;
      const int32_t* nu = side ? d->prod_nu : d->reac_nu;
      int order = 0, nsp = 0;
      for (int s = 0; s < 2; ++s) {
        const int k = idx[2 * i + s];
        if (k < 0) continue;
        if (k >= K) {
          snprintf(buf, sizeof buf, "reaction %d: species index %d out of range", i, k);
          return buf;
        }
        if (nu[2 * i + s] < 1 || nu[2 * i + s] > 2) {
          snprintf(buf, sizeof buf, "reaction %d: stoichiometric coefficient must be 1 or 2", i);
          return buf;
        }
        order += nu[2 * i + s];
        ++nsp;
      }
      if (nsp == 0 || order > 2) {
        snprintf(buf, sizeof buf, "reaction %d: each side needs 1..2 species of total order <= 2", i);
        return buf;
      }
      if (nsp == 2 && idx[2 * i] == idx[2 * i + 1]) {
        snprintf(buf, sizeof buf, "reaction %d: repeated species must use coefficient 2", i);
        return buf;
      }
    }
    for (int e = 0; e < E; ++e) {
      long bal = 0;
      for (int s = 0; s < 2; ++s) {
        if (d->reac_idx[2 * i + s] >= 0) bal -= (long)d->reac_nu[2 * i + s] * d->elem[d->reac_idx[2 * i + s] * E + e];
        if (d->prod_idx[2 * i + s] >= 0) bal += (long)d->prod_nu[2 * i + s] * d->elem[d->prod_idx[2 * i + s] * E + e];
      }
      if (bal != 0) {
        snprintf(buf, sizeof buf, "reaction %d: element %d not balanced", i, e);
        return buf;
      }
    }
    if (!(d->A[i] > 0.0) || !std::isfinite(d->b[i]) || !std::isfinite(d->Ea_R[i])) {
      snprintf(buf, sizeof buf, "reaction %d: need A > 0 and finite b, Ea_R", i);
      return buf;
    }
    if (t >= 2 && (!(d->A0[i] > 0.0) || !std::isfinite(d->b0[i]) || !std::isfinite(d->Ea0_R[i]))) {
      snprintf(buf, sizeof buf, "reaction %d: falloff needs A0 > 0 and finite b0, Ea0_R", i);
      return buf;
    }
    if (t == 3 && (!(d->troe[4 * i + 1] > 0.0) || !(d->troe[4 * i + 2] > 0.0) || !std::isfinite(d->troe[4 * i]))) {
      snprintf(buf, sizeof buf, "reaction %d: Troe needs T*** > 0 and T* > 0", i);
      return buf;
    }
    if (t >= 1)
      for (int k = 0; k < K; ++k)
        if (!std::isfinite(d->eff[(size_t)i * K + k]) || d->eff[(size_t)i * K + k] < 0.0) {
          snprintf(buf, sizeof buf, "reaction %d: efficiencies must be finite and >= 0", i);
          return buf;
        }
  }
  return "";
}

// ---------------------------------------------------------------------------
// device tables
// ---------------------------------------------------------------------------
namespace {

struct Pool {
  std::vector<unsigned char> host;
  size_t add(const void* src, size_t bytes) {
    size_t off = (host.size() + 255) & ~(size_t)255;
    host.resize(off + std::max<size_t>(bytes, 1));
    if (bytes) std::memcpy(host.data() + off, src, bytes);
    return off;
  }
};

}  // namespace

// The temperature below which some species may have |G/RT| > kBigGRT, from G/RT of
// every species on a 0.25 K grid over [kTmin, kTmax] with a threshold 10 below
// kBigGRT: by d(G/RT)/dT = -(H/RT)/T, |G/RT| changes by at most 0.25 |H/RT| / T
// between grid points, under 10 while |H/RT| < 40 T (8,000 at 200 K). A mechanism
// with a larger |H/RT| anywhere in the range always takes the one-exponential path.
// Returns 0 when no species comes near the threshold in the whole range.
static double big_gibbs_temperature(const chem_mechanism_desc* d) {
  const double thr = kBigGRT - 10.0;
  double Tb = 0.0;
  for (int k = 0; k < d->n_species; ++k) {
    bool found = false;
    for (double T = kTmax; T >= kTmin; T -= 0.25) {
      const double* a = (T < d->T_mid[k] ? d->nasa_lo : d->nasa_hi) + 7 * k;
      const double hrt = h_RT(a, T);
      if (!(std::fabs(hrt) < 40.0 * T)) return 1e300;
      if (!found && std::fabs(hrt - s_R(a, T)) > thr) {
        Tb = std::max(Tb, T + 0.25);
        found = true;
      }
    }
  }
  return Tb;
}

static chem_status build_tables(chem_handle h, const chem_mechanism_desc* d) {
  const int K = d->n_species, I = d->n_reactions;
  // sort reactions by kind so each warp meets at most a few kinds
  std::vector<int> order(I);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d->rxn_type[a] < d->rxn_type[b]; });
  h->rxn_order = order;
  std::vector<double> W(K), invW(K), nasa((size_t)36 * K, 0.0);
  for (int k = 0; k < K; ++k) {
    W[k] = d->W[k];
    invW[k] = 1.0 / d->W[k];
    for (int r = 0; r < 2; ++r) {
      const double* a = (r == 0 ? d->nasa_lo : d->nasa_hi) + 7 * k;
      double* o = &nasa[36 * k + 17 * r];
      for (int j = 0; j < 5; ++j) o[j] = a[j];
      o[5] = a[0];
      o[6] = a[1] / 2.0;
      o[7] = a[2] / 3.0;
      o[8] = a[3] / 4.0;
      o[9] = a[4] / 5.0;
      o[10] = a[5];
      o[11] = a[0];
      o[12] = a[1];
      o[13] = a[2] / 2.0;
      o[14] = a[3] / 3.0;
      o[15] = a[4] / 4.0;
      o[16] = a[6];
    }
    nasa[36 * k + 34] = d->T_mid[k];
  }
  // Each kind group is padded with null reactions to whole 32-reaction chunks, so a
  // warp's chunk never mixes kinds; chunks are dealt to warps by decreasing cost.
  std::vector<int> padded;
  std::vector<double> chunk_cost;  // estimated FP64 instructions of one rate evaluation
  for (int kind = 0; kind < 4; ++kind) {
    size_t first = padded.size();
    for (int i = 0; i < I; ++i)
      if (d->rxn_type[order[i]] == kind) padded.push_back(order[i]);
    if (padded.size() == first) continue;
    while (padded.size() % 32) padded.push_back(-1);
    const double cost = kind == 0 ? 28.0 : kind == 1 ? 31.0 : kind == 2 ? 60.0 : 220.0;
    for (size_t c = first; c < padded.size(); c += 32) chunk_cost.push_back(cost);
  }
  const int Ip = (int)padded.size();
  const int n_chunks = (int)chunk_cost.size();
  // Deal the chunks to warps, longest first, each to the warp with the least estimated
  // work so far; the species loops (thermo, production rates: ~72 per 32 species) load
  // the warps holding species and the CTA's scalar work (~60) the last warp.
  std::vector<int> by_cost(n_chunks);
  std::iota(by_cost.begin(), by_cost.end(), 0);
  std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return chunk_cost[a] > chunk_cost[b]; });
  std::vector<int> chunk_sched[3];
  for (int v = 0; v < 3; ++v) {
    const int NW = 2 << v, NT = 32 * NW;
    std::vector<double> load(NW, 0.0);
    for (int w = 0; w < NW; ++w) {
      int cnt = 0;
      for (int k = 0; k < K; ++k) cnt += (k % NT) / 32 == w;
      load[w] = 72.0 * ((cnt + 31) / 32);
    }
    load[NW - 1] += 60.0;
    std::vector<std::vector<int>> own(NW);
    for (int ch : by_cost) {
      int w = 0;
      for (int u = 1; u < NW; ++u)
        if (load[u] < load[w]) w = u;
      own[w].push_back(ch);
      load[w] += chunk_cost[ch];
    }
    chunk_sched[v].assign(1, 0);
    for (int w = 0; w < NW; ++w) chunk_sched[v].push_back(chunk_sched[v].back() + (int)own[w].size());
    for (int w = 0; w < NW; ++w) chunk_sched[v].insert(chunk_sched[v].end(), own[w].begin(), own[w].end());
  }
  h->rxn_order = padded;
  std::vector<double> arr((size_t)4 * std::max(Ip, 1), 0.0), fo, eff;
  std::vector<int4> slots(std::max(Ip, 1), make_int4(-1, -1, -1, -1));
  std::vector<int> rev(std::max(Ip, 1), 0);
  std::vector<std::vector<int2>> sp(K), tr(K);
  std::vector<std::vector<int4>> jr(K);
  int n_tb = 0, n_fo = 0, i_tb0 = Ip, i_fo0 = Ip, i_troe0 = Ip;
  // kind of each padded position (null entries take the kind of their group)
  std::vector<int> pkind(Ip);
  for (int i = 0, last = 0; i < Ip; ++i) {
    if (padded[i] >= 0) last = d->rxn_type[padded[i]];
    pkind[i] = last;
  }
  for (int i = 0; i < Ip; ++i) {
    const int o = padded[i];
    const int t = pkind[i];
    if (t >= 1 && i_tb0 == Ip) i_tb0 = i;
    if (t >= 2 && i_fo0 == Ip) i_fo0 = i;
    if (t == 3 && i_troe0 == Ip) i_troe0 = i;
    if (o < 0) {  // null reaction: zero rows keep the per-kind tables aligned
      if (t >= 1) {
        ++n_tb;
        eff.insert(eff.end(), K, 0.0);
      }
      if (t >= 2) {
        ++n_fo;
        fo.insert(fo.end(), 8, 0.0);
      }
      continue;
    }
    int sl[4] = {-1, -1, -1, -1};
    int dnu = 0;
    for (int side = 0; side < 2; ++side) {
      const int32_t* idx = side ? d->prod_idx : d->reac_idx;
      const int32_t* nu = side ? d->prod_nu : d->reac_nu;
      int w = 2 * side;
      for (int s = 0; s < 2; ++s) {
        const int k = idx[2 * o + s];
        if (k < 0) continue;
        for (int c = 0; c < nu[2 * o + s]; ++c) sl[w++] = k;
        dnu += side ? nu[2 * o + s] : -nu[2 * o + s];
      }
    }
    slots[i] = make_int4(sl[0], sl[1], sl[2], sl[3]);
    arr[4 * i + 0] = std::log(d->A[o]);
    arr[4 * i + 1] = d->b[o];
    arr[4 * i + 2] = d->Ea_R[o];
    arr[4 * i + 3] = (double)dnu;
    rev[i] = (d->reversible[o] ? 1 : 0) | ((dnu + 1) << 1);
    if (t >= 1) {
      ++n_tb;
      for (int k = 0; k < K; ++k) eff.push_back(d->eff[(size_t)o * K + k]);
    }
    if (t >= 2) {
      ++n_fo;
      const double* tr4 = d->troe + 4 * o;
      // Troe: reciprocal T*** and T* (Lindemann rows leave them unused)
      // low-pressure minus high-pressure Arrhenius parameters (k0 / kinf in one exp)
      const double f8[8] = {std::log(d->A0[o]) - std::log(d->A[o]), d->b0[o] - d->b[o], d->Ea0_R[o] - d->Ea_R[o], tr4[0],
                            t == 3 ? 1.0 / tr4[1] : 0.0, t == 3 ? 1.0 / tr4[2] : 0.0, tr4[3], 0.0};
      fo.insert(fo.end(), f8, f8 + 8);
    }
    // net stoichiometry per species
    std::vector<std::pair<int, int>> nets;
    for (int side = 0; side < 2; ++side) {
      const int32_t* idx = side ? d->prod_idx : d->reac_idx;
      const int32_t* nu = side ? d->prod_nu : d->reac_nu;
      for (int s = 0; s < 2; ++s) {
        const int k = idx[2 * o + s];
        if (k < 0) continue;
        const int v = side ? nu[2 * o + s] : -nu[2 * o + s];
        bool found = false;
        for (auto& pr : nets)
          if (pr.first == k) { pr.second += v; found = true; }
        if (!found) nets.push_back({k, v});
      }
    }
    for (auto& pr : nets) {
      if (pr.second == 0) continue;
      sp[pr.first].push_back(make_int2(i, pr.second));
      if (t >= 1) tr[pr.first].push_back(make_int2(i, pr.second));
      for (int s = 0; s < 4; ++s)
        if (sl[s] >= 0) jr[pr.first].push_back(make_int4(sl[s], i, pr.second, s));
    }
  }
  auto flatten2 = [&](std::vector<std::vector<int2>>& v, std::vector<int>& ptr, std::vector<int2>& ent) {
    ptr.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) ptr[k + 1] = ptr[k] + (int)v[k].size();
    for (int k = 0; k < K; ++k) ent.insert(ent.end(), v[k].begin(), v[k].end());
  };
  std::vector<int> sp_ptr, tr_ptr;
  std::vector<int2> sp_ent, tr_ent;
  flatten2(sp, sp_ptr, sp_ent);
  flatten2(tr, tr_ptr, tr_ent);
  // Mass-action Jacobian terms grouped by (row k, column j) pair in a fixed order,
  // then dealt to the threads of a CTA (longest pair first, to the thread with the
  // fewest terms so far, lowest thread on ties) for each block size.
  const int U = (K + 31) / 32, ldm = (K + 1) | 1;
  std::vector<unsigned> jmask((size_t)K * U, 0u);
  struct Pair {
    int k, j;
    std::vector<int2> ents;  // (4 i + slot, nu_ki)
  };
  std::vector<Pair> pairs;
  for (int k = 0; k < K; ++k) {
    std::vector<int4> ents = jr[k];  // (j, i, nu, slot)
    std::stable_sort(ents.begin(), ents.end(), [](const int4& a, const int4& b) { return a.x < b.x; });
    for (size_t e = 0; e < ents.size();) {
      Pair pr{k, ents[e].x, {}};
      for (; e < ents.size() && ents[e].x == pr.j; ++e) pr.ents.push_back(make_int2(4 * ents[e].y + ents[e].w, ents[e].z));
      jmask[(size_t)k * U + pr.j / 32] |= 1u << (pr.j % 32);
      pairs.push_back(std::move(pr));
    }
  }
  std::vector<int> by_len(pairs.size());
  std::iota(by_len.begin(), by_len.end(), 0);
  std::stable_sort(by_len.begin(), by_len.end(),
                   [&](int a, int b) { return pairs[a].ents.size() > pairs[b].ents.size(); });
  std::vector<int2> js_ent[3];
  std::vector<double> js_nu[3];
  int js_rounds[3];
  for (int v = 0; v < 3; ++v) {
    const int NT = 64 << v;
    std::vector<int> load(NT, 0);
    std::vector<std::vector<int>> own(NT);
    for (int q : by_len) {
      int t = 0;
      for (int u = 1; u < NT; ++u)
        if (load[u] < load[t]) t = u;
      own[t].push_back(q);
      load[t] += (int)pairs[q].ents.size();
    }
    const int R = std::max(1, *std::max_element(load.begin(), load.end()));
    js_rounds[v] = R;
    js_ent[v].assign((size_t)R * NT, make_int2(-1, -1));
    js_nu[v].assign((size_t)R * NT, 0.0);
    for (int t = 0; t < NT; ++t) {
      int r = 0;
      for (int q : own[t]) {
        const Pair& pr = pairs[q];
        for (size_t e = 0; e < pr.ents.size(); ++e, ++r) {
          const bool last = e + 1 == pr.ents.size();
          js_ent[v][(size_t)r * NT + t] = make_int2(pr.ents[e].x, last ? (1 + pr.k) * ldm + 1 + pr.j : -1);
          js_nu[v][(size_t)r * NT + t] = pr.ents[e].y * d->W[pr.k];
        }
      }
    }
  }

  std::vector<double> sp_nu(sp_ent.size()), tr_nu(tr_ent.size());
  for (size_t e = 0; e < sp_ent.size(); ++e) sp_nu[e] = sp_ent[e].y;
  for (int k = 0; k < K; ++k)
    for (int e = tr_ptr[k]; e < tr_ptr[k + 1]; ++e) tr_nu[e] = tr_ent[e].y * d->W[k];
  // float-float (hi, lo) copies of the constants the mixed form's assembly multiplies by
  auto split = [](const std::vector<double>& v) {
    std::vector<float> o(2 * v.size());
    for (size_t e = 0; e < v.size(); ++e) {
      const float h = (float)v[e];
      o[2 * e] = h;
      o[2 * e + 1] = (float)(v[e] - (double)h);
    }
    return o;
  };
  const std::vector<float> eff_ff = split(eff), invW_ff = split(invW), tr_nu_ff = split(tr_nu);
  // the efficiencies species-major as well: the rate evaluation's [M] sums read one
  // species for 32 consecutive reactions at a time (coalesced), the assembly one
  // reaction for 32 consecutive species
  std::vector<double> effT(eff.size());
  for (int r = 0; r < n_tb; ++r)
    for (int k = 0; k < K; ++k) effT[(size_t)k * n_tb + r] = eff[(size_t)r * K + k];
  const std::vector<float> effT_ff = split(effT);
  std::vector<float> js_nu_ff[3];
  for (int v = 0; v < 3; ++v) js_nu_ff[v] = split(js_nu[v]);
  Pool P;
  const size_t oW = P.add(W.data(), W.size() * 8), oiW = P.add(invW.data(), invW.size() * 8),
               oN = P.add(nasa.data(), nasa.size() * 8), oA = P.add(arr.data(), arr.size() * 8),
               oS = P.add(slots.data(), slots.size() * sizeof(int4)), oR = P.add(rev.data(), rev.size() * 4),
               oF = P.add(fo.data(), fo.size() * 8), oE = P.add(eff.data(), eff.size() * 8),
               oSp = P.add(sp_ptr.data(), sp_ptr.size() * 4), oSe = P.add(sp_ent.data(), sp_ent.size() * 8),
               oTp = P.add(tr_ptr.data(), tr_ptr.size() * 4), oTe = P.add(tr_ent.data(), tr_ent.size() * 8),
               oSn = P.add(sp_nu.data(), sp_nu.size() * 8), oTn = P.add(tr_nu.data(), tr_nu.size() * 8),
               oJm = P.add(jmask.data(), jmask.size() * 4),
               oEf = P.add(eff_ff.data(), eff_ff.size() * 4), oiWf = P.add(invW_ff.data(), invW_ff.size() * 4),
               oEt = P.add(effT.data(), effT.size() * 8), oEtf = P.add(effT_ff.data(), effT_ff.size() * 4),
               oTnf = P.add(tr_nu_ff.data(), tr_nu_ff.size() * 4);
  size_t oJe[3], oJn[3], oJnf[3], oCs[3];
  for (int v = 0; v < 3; ++v) {
    oCs[v] = P.add(chunk_sched[v].data(), chunk_sched[v].size() * 4);
    oJe[v] = P.add(js_ent[v].data(), js_ent[v].size() * sizeof(int2));
    oJn[v] = P.add(js_nu[v].data(), js_nu[v].size() * 8);
    oJnf[v] = P.add(js_nu_ff[v].data(), js_nu_ff[v].size() * 4);
  }
  CHEM_CUDA(h, cudaMalloc(&h->d_tables, P.host.size()));
  CHEM_CUDA(h, cudaMemcpy(h->d_tables, P.host.data(), P.host.size(), cudaMemcpyHostToDevice));
  unsigned char* b = static_cast<unsigned char*>(h->d_tables);
  DevMech& m = h->dm;
  m.K = K;
  m.I = Ip;
  m.n_chunks = n_chunks;
  h->I = std::max(Ip, 1);
  m.n_tb = n_tb;
  m.n_fo = n_fo;
  m.i_tb0 = i_tb0;
  m.i_fo0 = i_fo0;
  m.i_troe0 = i_troe0;
  m.T_bigG = big_gibbs_temperature(d);
  m.W = reinterpret_cast<const double*>(b + oW);
  m.invW = reinterpret_cast<const double*>(b + oiW);
  m.nasa = reinterpret_cast<const double*>(b + oN);
  m.arr = reinterpret_cast<const double*>(b + oA);
  m.slots = reinterpret_cast<const int4*>(b + oS);
  m.rev = reinterpret_cast<const int*>(b + oR);
  m.fo = reinterpret_cast<const double*>(b + oF);
  m.eff = reinterpret_cast<const double*>(b + oE);
  m.sp_ptr = reinterpret_cast<const int*>(b + oSp);
  m.sp_ent = reinterpret_cast<const int2*>(b + oSe);
  m.tr_ptr = reinterpret_cast<const int*>(b + oTp);
  m.tr_ent = reinterpret_cast<const int2*>(b + oTe);
  m.sp_nu = reinterpret_cast<const double*>(b + oSn);
  m.tr_nu = reinterpret_cast<const double*>(b + oTn);
  m.eff_ff = reinterpret_cast<const chem::ff2*>(b + oEf);
  m.effT = reinterpret_cast<const double*>(b + oEt);
  m.effT_ff = reinterpret_cast<const chem::ff2*>(b + oEtf);
  m.invW_ff = reinterpret_cast<const chem::ff2*>(b + oiWf);
  m.tr_nu_ff = reinterpret_cast<const chem::ff2*>(b + oTnf);
  m.jmask = reinterpret_cast<const unsigned*>(b + oJm);
  for (int v = 0; v < 3; ++v) {
    m.js_ent[v] = reinterpret_cast<const int2*>(b + oJe[v]);
    m.js_nu[v] = reinterpret_cast<const double*>(b + oJn[v]);
    m.js_nu_ff[v] = reinterpret_cast<const chem::ff2*>(b + oJnf[v]);
    m.js_rounds[v] = js_rounds[v];
    m.chunk_sched[v] = reinterpret_cast<const int*>(b + oCs[v]);
  }
  return CHEM_OK;
}

// ---------------------------------------------------------------------------
// handle lifecycle
// ---------------------------------------------------------------------------
extern "C" chem_status chem_create(const chem_mechanism_desc* desc, chem_handle* out) {
  if (!desc || !out) {
    g_create_error = "chem_create: NULL argument";
    return CHEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::string v = validate(desc);
  if (!v.empty()) {
    g_create_error = "chem_create: " + v;
    return CHEM_ERR_BAD_MECHANISM;
  }
  chem_handle h = new chem_handle_s();
  h->K = desc->n_species;
  h->I = desc->n_reactions;
  h->I_user = desc->n_reactions;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    g_create_error = cuda_msg("chem_create", e);
    delete h;
    return CHEM_ERR_CUDA;
  }
  h->n_elem = desc->n_elements;
  if (desc->n_elements > 0)
    h->elem_host.assign(desc->elem, desc->elem + (size_t)desc->n_species * desc->n_elements);
  h->W_host.assign(desc->W, desc->W + desc->n_species);
  chem_status s = build_tables(h, desc);
  if (s == CHEM_OK) s = chem_internal_alloc(h, &h->d_queue, sizeof(int) * 4);
  if (s != CHEM_OK) {
    g_create_error = h->err;
    chem_destroy(h);
    return s;
  }
  *out = h;
  return CHEM_OK;
}

extern "C" chem_status chem_destroy(chem_handle h) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  chem_internal_release_learned(h);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->kev0) cudaEventDestroy(h->kev0);
  if (h->kev1) cudaEventDestroy(h->kev1);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (void* p : h->allocations) cudaFree(p);
  if (h->d_tables) cudaFree(h->d_tables);
  delete h;
  return CHEM_OK;
}

chem_status chem_internal_alloc(chem_handle h, void* pp, size_t bytes) {
  void** p = reinterpret_cast<void**>(pp);
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    h->err = cuda_msg("cudaMalloc", e);
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? CHEM_ERR_OOM : CHEM_ERR_CUDA;
  }
  h->allocations.push_back(*p);
  return CHEM_OK;
}

static void release(chem_handle h, void* p) {
  if (!p) return;
  auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
  if (it != h->allocations.end()) h->allocations.erase(it);
  cudaFree(p);
}

// Per-cell statistics buffers sized for n cells.
static chem_status ensure_stats(chem_handle h, int64_t n) {
  if (n <= h->stats_cap) return CHEM_OK;
  cudaDeviceSynchronize();
  release(h, h->d_sub);
  release(h, h->d_rej);
  release(h, h->d_status);
  release(h, h->d_hfirst);
  release(h, h->d_hlast);
  release(h, h->d_cost);
  h->d_sub = h->d_rej = h->d_status = nullptr;
  h->d_hfirst = h->d_hlast = nullptr;
  h->hlast_valid = false;
  h->d_cost = nullptr;
  h->stats_cap = 0;
  const int64_t cap = std::max<int64_t>(n, 1024);
  chem_status s;
  if ((s = chem_internal_alloc(h, &h->d_sub, cap * 4)) != CHEM_OK) return s;
  if ((s = chem_internal_alloc(h, &h->d_rej, cap * 4)) != CHEM_OK) return s;
  if ((s = chem_internal_alloc(h, &h->d_status, cap * 4)) != CHEM_OK) return s;
  if ((s = chem_internal_alloc(h, &h->d_hfirst, cap * 8)) != CHEM_OK) return s;
  if ((s = chem_internal_alloc(h, &h->d_hlast, cap * 8)) != CHEM_OK) return s;
  if ((s = chem_internal_alloc(h, &h->d_cost, cap * 4)) != CHEM_OK) return s;
  h->stats_cap = cap;
  h->cost_valid = false;
  return CHEM_OK;
}

// ---------------------------------------------------------------------------
// options
// ---------------------------------------------------------------------------
struct OptionDef {
  const char* key;
  int chem_handle_s::*field;
  double lo, hi;
};
static const OptionDef kOptions[] = {
    {"precision", &chem_handle_s::precision, 0, 2},
    {"ir_sweeps", &chem_handle_s::ir_sweeps, 0, 3},
    {"scheduler", &chem_handle_s::scheduler, 0, 2},
    {"order", &chem_handle_s::order, 0, 2},
    {"h0", &chem_handle_s::h0mode, 0, 2},
    {"max_steps", &chem_handle_s::max_steps, 1, 2147483647.0},
    {"block", &chem_handle_s::block, 0, 256},
    {"ctas_per_sm", &chem_handle_s::ctas_per_sm, 0, 64},
    {"graph", &chem_handle_s::graph, 0, 1},
    {"autotune", &chem_handle_s::autotune, 0, 1},
    {"profile", &chem_handle_s::profile, 0, 1},
    {"time_kernel", &chem_handle_s::time_kernel, 0, 1},
    {"jacobian", &chem_handle_s::jac_fd, 0, 1},
    {"pivoting", &chem_handle_s::pivoting, 0, 1},
    {"job_launch", &chem_handle_s::job_launch, 0, 1},
    {"method", &chem_handle_s::method, 0, 1},
    {"h0_guard", &chem_handle_s::h0_guard, 0, 1},
    {"h0_range", &chem_handle_s::h0_range, 0, 1000},
};

extern "C" chem_status chem_set_option(chem_handle h, const char* key, double value) {
  if (!h || !key) return CHEM_ERR_INVALID_ARG;
  for (const auto& o : kOptions) {
    if (std::strcmp(o.key, key) != 0) continue;
    if (!(value >= o.lo && value <= o.hi) || value != std::floor(value)) {
      h->err = std::string("chem_set_option: value out of range for ") + key;
      return CHEM_ERR_INVALID_ARG;
    }
    if (std::strcmp(key, "block") == 0 && value != 0 && value != 64 && value != 128 && value != 256) {
      h->err = "chem_set_option: block must be 0 (automatic), 64, 128 or 256";
      return CHEM_ERR_INVALID_ARG;
    }
    h->*(o.field) = (int)value;
    if (std::strcmp(key, "block") == 0 || std::strcmp(key, "precision") == 0 || std::strcmp(key, "method") == 0)
      h->autotuned_key = -1;  // explicit choice wins; a new kernel is tuned afresh
    return CHEM_OK;
  }
  h->err = std::string("chem_set_option: unknown key ") + key;
  return CHEM_ERR_INVALID_ARG;
}

extern "C" chem_status chem_get_option(chem_handle h, const char* key, double* value) {
  if (!h || !key || !value) return CHEM_ERR_INVALID_ARG;
  if (std::strcmp(key, "last_block") == 0) {  // read-only: threads per CTA of the last launch
    *value = (double)h->last_block;
    return CHEM_OK;
  }
  for (const auto& o : kOptions)
    if (std::strcmp(o.key, key) == 0) {
      *value = (double)(h->*(o.field));
      return CHEM_OK;
    }
  h->err = std::string("chem_get_option: unknown key ") + key;
  return CHEM_ERR_INVALID_ARG;
}

extern "C" const char* chem_last_error(chem_handle h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}
extern "C" int32_t chem_n_species(chem_handle h) { return h ? h->K : -1; }
extern "C" int32_t chem_n_reactions(chem_handle h) { return h ? h->I_user : -1; }

// ---------------------------------------------------------------------------
// integration
// ---------------------------------------------------------------------------
static bool bad_tol(double dt, double rtol, double atol) { return chem_internal_bad_tol(dt, rtol, atol); }

chem_status chem_internal_integrate(const chem_job* jobs, int32_t n_jobs, double dt, double rtol,
                                    double atol, cudaStream_t st) {
  chem_handle h0 = jobs[0].h;
  bool rm = false;  // reference mapping (one job, queue scheduler)
  for (int j = 0; j < n_jobs; ++j) {
    rm = rm || jobs[j].h->refmap;
    jobs[j].h->rm_last_n = -1;
    jobs[j].h->noalloc_n = -1;
  }
  if (rm && (n_jobs != 1 || h0->scheduler != SCHED_QUEUE)) {
    h0->err = "chem_integrate: reference mapping needs one job and the queue scheduler";
    return CHEM_ERR_INVALID_ARG;
  }
  IntegrateArgs a;
  std::memset(&a, 0, sizeof a);
  int64_t total = 0;
  int Kmax = 0, Imax = 0;
  for (int j = 0; j < n_jobs; ++j) {
    chem_handle h = jobs[j].h;
    chem_status s = ensure_stats(h, jobs[j].n_cells);
    if (s != CHEM_OK) {
      h0->err = h->err;
      return s;
    }
    Job& J = a.jobs[j];
    J.m = h->dm;
    J.n_cells = jobs[j].n_cells;
    J.offset = total;
    J.T = jobs[j].T;
    J.p = jobs[j].p;
    J.Y = jobs[j].Y;
    J.st.substeps = h->d_sub;
    J.st.rejects = h->d_rej;
    J.st.h_first = h->d_hfirst;
    J.st.status = h->d_status;
    J.cost_out = h->d_cost;
    J.st.h_last = h->d_hlast;
    // carried-over initial steps: the previous call's proposals for the same cells
    // (read at a cell's start, overwritten at its end by the same CTA)
    J.h0 = (h->h0mode == 2 && h->hlast_valid && h->hlast_n == jobs[j].n_cells) ? h->d_hlast : nullptr;
    if (J.h0) a.use_h0 = 1;
    h->last_n = jobs[j].n_cells;
    total += jobs[j].n_cells;
    Kmax = std::max(Kmax, h->K);
    Imax = std::max(Imax, h->I);
  }
  if (total == 0) return CHEM_OK;
  if (total > 2147483647LL) {
    h0->err = "chem_integrate: more than 2^31-1 cells in one call";
    return CHEM_ERR_INVALID_ARG;
  }
  a.n_jobs = n_jobs;
  a.n_total = total;
  a.dt = dt;
  a.rtol = rtol;
  a.atol = atol;
  a.max_steps = h0->max_steps;
  a.sched = h0->scheduler;
  a.ir_sweeps = h0->ir_sweeps;
  a.jac_fd = h0->jac_fd;
  a.no_pivot = h0->pivoting ? 0 : 1;
  a.smem_K = Kmax;
  a.smem_I = std::max(Imax, 1);
  a.queue = static_cast<int*>(h0->d_queue);
  a.perm = nullptr;
  a.phase = nullptr;
  a.tab = method_tableau(h0->method);
  a.h0_guard = h0->h0_guard;
  if (h0->profile) {
    if (!h0->d_phase) {
      chem_status ps = chem_internal_alloc(h0, &h0->d_phase, 8 * sizeof(unsigned long long));
      if (ps != CHEM_OK) return ps;
      CHEM_CUDA(h0, cudaMemsetAsync(h0->d_phase, 0, 8 * sizeof(unsigned long long), st));
    }
    a.phase = h0->d_phase;
  }
  chem_status s = chem_internal_prepare_learned(h0, jobs, n_jobs, &a, st);
  if (s != CHEM_OK) return s;
  const size_t smem = smem_bytes(a.smem_K, a.smem_I, h0->precision);
  if (smem > 227 * 1024) {
    h0->err = "chem_integrate: mechanism too large for shared memory";
    return CHEM_ERR_INVALID_ARG;
  }
  // the mixed form may keep its assembled matrix in global memory on persistent grids when
  // that lets more CTAs share an SM (large mechanisms)
  const bool m0g_ok = h0->precision == PREC_MIXED && a.sched != SCHED_PLAIN;
  int block = h0->block ? h0->block : chem_internal_pick_block(h0, a.smem_K, a.smem_I, m0g_ok);
  int tuned_ctas = 0, tuned_m0g = -1;  // the autotuner's resident CTAs per SM and matrix layout
  if (h0->autotune) {
    s = chem_internal_autotune(h0, a, st, &block, &tuned_ctas, &tuned_m0g);
    if (s != CHEM_OK) return s;
  }
  h0->last_block = block;
  int grid;
  if (a.sched == SCHED_PLAIN) {
    grid = (int)total;
  } else {
    int occ = 0;
    CHEM_CUDA(h0, occupancy_integrate(block, h0->precision, a.smem_K, a.smem_I, &occ));
    bool m0g = false;
    if (m0g_ok) {
      int occ_g = 0;
      CHEM_CUDA(h0, occupancy_integrate(block, h0->precision, a.smem_K, a.smem_I, &occ_g, true));
      if (tuned_m0g >= 0 ? tuned_m0g == 1 : occ_g > occ) {
        occ = occ_g;
        m0g = true;
      }
    }
    if (tuned_ctas > 0) occ = std::min(occ, tuned_ctas);
    if (occ < 1) {
      h0->err = "chem_integrate: kernel does not fit on an SM";
      return CHEM_ERR_CUDA;
    }
    if (h0->ctas_per_sm > 0) occ = std::min(occ, h0->ctas_per_sm);
    grid = (int)std::min<int64_t>(total, (int64_t)occ * h0->num_sms);
    if (m0g) {
      const int nmax = a.smem_K + 1;
      const int64_t stride = (int64_t)nmax * (nmax | 1);
      const size_t bytes = (size_t)grid * stride * sizeof(double);
      if (bytes > h0->m0_cap) {
        cudaStreamSynchronize(st);
        if (h0->d_m0) {
          release(h0, h0->d_m0);
          h0->d_m0 = nullptr;
          h0->m0_cap = 0;
        }
        s = chem_internal_alloc(h0, &h0->d_m0, bytes);
        if (s != CHEM_OK) return s;
        h0->m0_cap = bytes;
      }
      a.m0_scratch = h0->d_m0;
      a.m0_stride = stride;
    }
  }
  // reference mapping: mapped cells go to the front of the work order and the
  // queue starts past them; after the launch they take the reference's change
  if (rm) {
    s = chem_internal_refmap_prepare(h0, jobs[0], &a, st);
    if (s != CHEM_OK) return s;
  }
  s = chem_internal_launch(h0, a, block, grid, st);
  h0->queue_preset = false;
  if (s != CHEM_OK) return s;
  if (rm) {
    s = chem_internal_refmap_apply(h0, jobs[0], st);
    if (s != CHEM_OK) return s;
  }
  for (int j = 0; j < n_jobs; ++j) {
    jobs[j].h->cost_valid = true;
    jobs[j].h->cost_n = jobs[j].n_cells;
    jobs[j].h->hlast_valid = true;
    jobs[j].h->hlast_n = jobs[j].n_cells;
  }
  return CHEM_OK;
}

// Block size with the most resident warps per SM for this mechanism size and
// precision (ties: 128, then 64, then 256 threads).
int chem_internal_pick_block(chem_handle h, int K, int I, bool allow_m0_global) {
  int best = 128, best_w = -1;
  for (int b : {128, 64, 256}) {
    int occ = 0;
    if (occupancy_integrate(b, h->precision, K, I, &occ) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    int occ_g = 0;
    if (allow_m0_global && occupancy_integrate(b, h->precision, K, I, &occ_g, true) == cudaSuccess)
      occ = std::max(occ, occ_g);
    cudaGetLastError();
    if (occ * b / 32 > best_w) {
      best_w = occ * b / 32;
      best = b;
    }
  }
  return best;
}

// Launch (optionally through a cached CUDA graph).
chem_status chem_internal_launch(chem_handle h, const IntegrateArgs& a, int block, int grid, cudaStream_t st) {
  if (h->time_kernel && !h->kev0) {
    CHEM_CUDA(h, cudaEventCreate(&h->kev0));
    CHEM_CUDA(h, cudaEventCreate(&h->kev1));
  }
  if (h->graph) {
    if (h->time_kernel) CHEM_CUDA(h, cudaEventRecord(h->kev0, st));
    chem_status s = chem_internal_graph_launch(h, a, block, grid, st);
    if (s != CHEM_OK) return s;
  } else {
    if (a.sched == SCHED_QUEUE && !h->queue_preset) CHEM_CUDA(h, cudaMemsetAsync(a.queue, 0, sizeof(int), st));
    if (h->time_kernel) CHEM_CUDA(h, cudaEventRecord(h->kev0, st));
    CHEM_CUDA(h, launch_integrate(a, block, h->precision, grid, st));
  }
  if (h->time_kernel) {
    CHEM_CUDA(h, cudaEventRecord(h->kev1, st));
    h->kev_recorded = true;
  }
  return CHEM_OK;
}

extern "C" chem_status chem_get_kernel_ms(chem_handle h, float* ms) {
  if (!h || !ms) return CHEM_ERR_INVALID_ARG;
  if (!h->kev_recorded) {
    h->err = "chem_get_kernel_ms: no integration launch was timed (option time_kernel)";
    return CHEM_ERR_INVALID_ARG;
  }
  CHEM_CUDA(h, cudaEventSynchronize(h->kev1));
  CHEM_CUDA(h, cudaEventElapsedTime(ms, h->kev0, h->kev1));
  return CHEM_OK;
}

extern "C" chem_status chem_integrate(chem_handle h, int64_t n_cells, double* T, const double* p, double* Y,
                                      double dt, double rtol, double atol, void* stream) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  if (n_cells < 0 || (n_cells > 0 && (!T || !p || !Y)) || bad_tol(dt, rtol, atol)) {
    h->err = "chem_integrate: invalid argument (n_cells < 0, NULL array, or dt/rtol/atol out of range)";
    return CHEM_ERR_INVALID_ARG;
  }
  chem_job j{h, n_cells, T, p, Y};
  return chem_internal_integrate(&j, 1, dt, rtol, atol, static_cast<cudaStream_t>(stream));
}

// Option job_launch = 1: one integration launch per job, each with its own handle's
// options (block size and shared-memory layout fitted to its mechanism), on the
// handles' own streams forked from and joined back into the caller's stream by
// events, so that the kernels may run concurrently and a later job's CTAs fill the
// SMs an earlier job's tail leaves idle.
static chem_status integrate_jobs_concurrent(const chem_job* jobs, int32_t n_jobs, double dt, double rtol,
                                             double atol, cudaStream_t st) {
  chem_handle h0 = jobs[0].h;
  for (int j = 0; j < n_jobs; ++j) {
    chem_handle h = jobs[j].h;
    if (!h->side) {
      CHEM_CUDA(h0, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
      CHEM_CUDA(h0, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
      CHEM_CUDA(h0, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
  }
  CHEM_CUDA(h0, cudaEventRecord(h0->ev_fork, st));
  chem_status s = CHEM_OK;
  bool joined[kMaxJobs] = {};
  for (int j = 0; j < n_jobs && s == CHEM_OK; ++j) {
    chem_handle h = jobs[j].h;
    cudaError_t e = cudaStreamWaitEvent(h->side, h0->ev_fork, 0);
    if (e != cudaSuccess) {
      h0->err = cuda_msg("cudaStreamWaitEvent", e);
      s = CHEM_ERR_CUDA;
      break;
    }
    s = chem_internal_integrate(&jobs[j], 1, dt, rtol, atol, h->side);
    if (s != CHEM_OK && h != h0) h0->err = h->err;
    // joined even after an error, so that the caller's stream orders after all enqueued work
    joined[j] = cudaEventRecord(h->ev_join, h->side) == cudaSuccess;
  }
  for (int j = 0; j < n_jobs; ++j) {
    if (!joined[j]) continue;
    cudaError_t e = cudaStreamWaitEvent(st, jobs[j].h->ev_join, 0);
    if (e != cudaSuccess && s == CHEM_OK) {
      h0->err = cuda_msg("cudaStreamWaitEvent", e);
      s = CHEM_ERR_CUDA;
    }
  }
  return s;
}

extern "C" chem_status chem_integrate_jobs(const chem_job* jobs, int32_t n_jobs, double dt, double rtol,
                                           double atol, void* stream) {
  if (!jobs || n_jobs < 1 || n_jobs > kMaxJobs || !jobs[0].h) return CHEM_ERR_INVALID_ARG;
  chem_handle h0 = jobs[0].h;
  if (bad_tol(dt, rtol, atol)) {
    h0->err = "chem_integrate_jobs: dt/rtol/atol out of range";
    return CHEM_ERR_INVALID_ARG;
  }
  for (int j = 0; j < n_jobs; ++j) {
    if (!jobs[j].h || jobs[j].n_cells < 0 || (jobs[j].n_cells > 0 && (!jobs[j].T || !jobs[j].p || !jobs[j].Y))) {
      h0->err = "chem_integrate_jobs: invalid job";
      return CHEM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < j; ++i)
      if (jobs[i].h == jobs[j].h) {
        h0->err = "chem_integrate_jobs: each job needs its own handle";
        return CHEM_ERR_INVALID_ARG;
      }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h0->job_launch == 1 && n_jobs > 1) return integrate_jobs_concurrent(jobs, n_jobs, dt, rtol, atol, st);
  return chem_internal_integrate(jobs, n_jobs, dt, rtol, atol, st);
}

extern "C" chem_status chem_integrate_host(chem_handle h, int64_t n_cells, double* T, const double* p,
                                           double* Y, double dt, double rtol, double atol, void* stream) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  if (n_cells < 0 || (n_cells > 0 && (!T || !p || !Y)) || bad_tol(dt, rtol, atol)) {
    h->err = "chem_integrate_host: invalid argument";
    return CHEM_ERR_INVALID_ARG;
  }
  if (n_cells == 0) return CHEM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_cells > h->stage_cap) {
    CHEM_CUDA(h, cudaStreamSynchronize(st));
    release(h, h->d_stage);
    h->d_stage = nullptr;
    h->stage_cap = 0;
    chem_status s = chem_internal_alloc(h, &h->d_stage, (size_t)n_cells * (h->K + 2) * sizeof(double));
    if (s != CHEM_OK) return s;
    h->stage_cap = n_cells;
  }
  double* dT = static_cast<double*>(h->d_stage);
  double* dp = dT + n_cells;
  double* dY = dp + n_cells;
  const size_t nY = (size_t)n_cells * h->K * sizeof(double);
  CHEM_CUDA(h, cudaMemcpyAsync(dT, T, n_cells * sizeof(double), cudaMemcpyHostToDevice, st));
  CHEM_CUDA(h, cudaMemcpyAsync(dp, p, n_cells * sizeof(double), cudaMemcpyHostToDevice, st));
  CHEM_CUDA(h, cudaMemcpyAsync(dY, Y, nY, cudaMemcpyHostToDevice, st));
  chem_status s = chem_integrate(h, n_cells, dT, dp, dY, dt, rtol, atol, stream);
  if (s != CHEM_OK) return s;
  CHEM_CUDA(h, cudaMemcpyAsync(T, dT, n_cells * sizeof(double), cudaMemcpyDeviceToHost, st));
  CHEM_CUDA(h, cudaMemcpyAsync(Y, dY, nY, cudaMemcpyDeviceToHost, st));
  CHEM_CUDA(h, cudaStreamSynchronize(st));
  return CHEM_OK;
}

// ---------------------------------------------------------------------------
// statistics
// ---------------------------------------------------------------------------
chem_status chem_internal_stats_view(chem_handle h, chem_stats_view* v) {
  if (h->noalloc_n >= 0) return chem_internal_noalloc_stats(h, h->noalloc_n, v);
  v->n = h->last_n;
  v->substeps = h->d_sub;
  v->rejects = h->d_rej;
  v->status = h->d_status;
  v->h_first = h->d_hfirst;
  return CHEM_OK;
}

extern "C" chem_status chem_get_stats(chem_handle h, void* stream, int32_t* substeps, int32_t* rejects,
                                      double* h_first, int32_t* cell_status) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  chem_stats_view v;
  chem_status vs = chem_internal_stats_view(h, &v);
  if (vs != CHEM_OK) return vs;
  const int64_t n = v.n;
  if (n == 0) return CHEM_OK;
  if (substeps) CHEM_CUDA(h, cudaMemcpyAsync(substeps, v.substeps, n * 4, cudaMemcpyDeviceToDevice, st));
  if (rejects) CHEM_CUDA(h, cudaMemcpyAsync(rejects, v.rejects, n * 4, cudaMemcpyDeviceToDevice, st));
  if (h_first) CHEM_CUDA(h, cudaMemcpyAsync(h_first, v.h_first, n * 8, cudaMemcpyDeviceToDevice, st));
  if (cell_status) CHEM_CUDA(h, cudaMemcpyAsync(cell_status, v.status, n * 4, cudaMemcpyDeviceToDevice, st));
  std::vector<int32_t> hs(n);
  CHEM_CUDA(h, cudaMemcpyAsync(hs.data(), v.status, n * 4, cudaMemcpyDeviceToHost, st));
  CHEM_CUDA(h, cudaStreamSynchronize(st));
  for (int64_t i = 0; i < n; ++i)
    if (hs[i] != CHEM_CELL_OK) {
      h->err = "chem_get_stats: some cells failed (see cell_status)";
      return CHEM_ERR_CELLS_FAILED;
    }
  return CHEM_OK;
}

extern "C" chem_status chem_get_totals(chem_handle h, void* stream, int64_t* n_cells, int64_t* substeps,
                                       int64_t* rejects, int64_t* failed) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  chem_stats_view v;
  chem_status vs = chem_internal_stats_view(h, &v);
  if (vs != CHEM_OK) return vs;
  const int64_t n = v.n;
  std::vector<int32_t> a(n), b(n), c(n);
  if (n > 0) {
    CHEM_CUDA(h, cudaMemcpyAsync(a.data(), v.substeps, n * 4, cudaMemcpyDeviceToHost, st));
    CHEM_CUDA(h, cudaMemcpyAsync(b.data(), v.rejects, n * 4, cudaMemcpyDeviceToHost, st));
    CHEM_CUDA(h, cudaMemcpyAsync(c.data(), v.status, n * 4, cudaMemcpyDeviceToHost, st));
  }
  CHEM_CUDA(h, cudaStreamSynchronize(st));
  int64_t s1 = 0, s2 = 0, s3 = 0;
  for (int64_t i = 0; i < n; ++i) {
    s1 += a[i];
    s2 += b[i];
    s3 += c[i] != CHEM_CELL_OK;
  }
  if (n_cells) *n_cells = n;
  if (substeps) *substeps = s1;
  if (rejects) *rejects = s2;
  if (failed) *failed = s3;
  return CHEM_OK;
}

// ---------------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------------
extern "C" chem_status chem_get_phase_cycles(chem_handle h, void* stream, uint64_t* cycles, int32_t reset) {
  if (!h || !cycles) return CHEM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < 8; ++k) cycles[k] = 0;
  if (!h->d_phase) return CHEM_OK;
  CHEM_CUDA(h, cudaMemcpyAsync(cycles, h->d_phase, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  if (reset) CHEM_CUDA(h, cudaMemsetAsync(h->d_phase, 0, 8 * sizeof(uint64_t), st));
  CHEM_CUDA(h, cudaStreamSynchronize(st));
  return CHEM_OK;
}

extern "C" chem_status chem_eval_rhs(chem_handle h, int64_t n, const double* T, const double* p,
                                     const double* Y, double* f, void* stream) {
  if (!h || n < 0 || (n > 0 && (!T || !p || !Y || !f))) return CHEM_ERR_INVALID_ARG;
  if (n == 0) return CHEM_OK;
  CHEM_CUDA(h, launch_diag(h->dm, n, T, p, Y, f, 0, 0, 0, 0, h->precision, static_cast<cudaStream_t>(stream)));
  return CHEM_OK;
}

extern "C" chem_status chem_eval_jacobian(chem_handle h, int64_t n, const double* T, const double* p,
                                          const double* Y, double* J, void* stream) {
  if (!h || n < 0 || (n > 0 && (!T || !p || !Y || !J))) return CHEM_ERR_INVALID_ARG;
  if (n == 0) return CHEM_OK;
  CHEM_CUDA(h, launch_diag(h->dm, n, T, p, Y, J, 0, 0, 0, 1, h->precision, static_cast<cudaStream_t>(stream),
                           h->jac_fd));
  return CHEM_OK;
}

extern "C" chem_status chem_eval_h0(chem_handle h, int64_t n, const double* T, const double* p, const double* Y,
                                    double dt, double rtol, double atol, double* h0, void* stream) {
  if (!h || n < 0 || (n > 0 && (!T || !p || !Y || !h0)) || bad_tol(dt, rtol, atol)) return CHEM_ERR_INVALID_ARG;
  if (n == 0) return CHEM_OK;
  CHEM_CUDA(h, launch_diag(h->dm, n, T, p, Y, h0, dt, rtol, atol, 2, h->precision, static_cast<cudaStream_t>(stream),
                           0, method_tableau(h->method).q));
  return CHEM_OK;
}

extern "C" chem_status chem_lu_solve_batched(int64_t n_mat, int32_t dim, const double* A, const double* b,
                                             double* x, int32_t* info, int32_t precision, int32_t ir_sweeps,
                                             void* stream) {
  if (n_mat < 0 || dim < 1 || dim > 128 || precision < 0 || precision > 2 || ir_sweeps < 0 || ir_sweeps > 3)
    return CHEM_ERR_INVALID_ARG;
  if (n_mat == 0) return CHEM_OK;
  if (!A || !b || !x) return CHEM_ERR_INVALID_ARG;
  cudaError_t e = launch_lu_solve(n_mat, dim, A, b, x, info, precision, ir_sweeps, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? CHEM_OK : CHEM_ERR_CUDA;
}

extern "C" chem_status chem_eval_math(int32_t op, int64_t n, const double* x, double* y, void* stream) {
  if (op < 0 || op > 4 || n < 0 || (n > 0 && (!x || !y))) return CHEM_ERR_INVALID_ARG;
  return launch_math(op, x, y, n, static_cast<cudaStream_t>(stream)) == cudaSuccess ? CHEM_OK : CHEM_ERR_CUDA;
}

extern "C" void chem_rosenbrock_tableau(double* gamma, double* a, double* c, double* m, double* e) {
  if (gamma) *gamma = kRodasGamma;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) {
      if (a) a[6 * i + j] = kRodasA[i][j];
      if (c) c[6 * i + j] = kRodasC[i][j];
    }
    if (m) m[i] = kRodasM[i];
    if (e) e[i] = kRodasE[i];
  }
}

extern "C" int32_t chem_method_tableau(int32_t method, double* gamma, double* a, double* c, double* m, double* e) {
  if (method < 0 || method > 1) return -1;
  const MethodTab t = method_tableau(method);
  if (gamma) *gamma = t.gamma;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) {
      if (a) a[6 * i + j] = t.a[i][j];
      if (c) c[6 * i + j] = t.c[i][j];
    }
    if (m) m[i] = t.m[i];
    if (e) e[i] = t.e[i];
  }
  return t.s;
}
