// C ABI of libtnlbm: the simulation object (one MPS-LBM time step captured as
// a CUDA graph) and the batched MPS primitives.
//
// The step (Sec. 3.2) is written as a DAG of MPS nodes; every node is produced
// by a rounding job (a rounded linear combination of exactly formed terms) or a
// product fit (Sec. 2.3).  Jobs are grouped by dependency level; a level runs
// its rounding jobs in one launch and its fits on a second stream, so the
// whole step is a fork-join graph.  Order of the linear combinations:
//   a1 moments as balanced pairwise trees; a6 shared prefix sums
//   E0 = ((rho - 1.5 Pxx) - 1.5 Pyy) - 1.5 Pzz, second-order prefixes (diagonal
//   terms xx, yy, zz first, then xy, xz, yz), sign-normalised first-order sums;
//   a7 one axis shift at a time (x, y, z) with the bounce-back term added in the
//   last rounding; a8 g_i = f_i . m_O used in both object terms, and the object
//   update (f_i - g_i) + S g_opp(i) as two pairwise rounded sums.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "fit.cuh"
#include "internal.cuh"

namespace tn {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
  return TNLBM_E_CUDA;
}

// ---------------------------------------------------------------- lattices
struct LatticeDef {
  int Q;
  int c[19][3];
  double w[19];
  int opp[19];
};

static LatticeDef make_lattice(int q) {
  LatticeDef L{};
  static const int c19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                 {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                 {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                 {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
  static const int c15[15][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                 {0, 0, 1},  {0, 0, -1},  {1, 1, 1},  {-1, -1, -1}, {1, 1, -1},
                                 {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
  L.Q = q;
  for (int i = 0; i < q; ++i) {
    for (int d = 0; d < 3; ++d) L.c[i][d] = (q == 19) ? c19[i][d] : c15[i][d];
    if (q == 19) L.w[i] = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    else L.w[i] = i == 0 ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
    L.opp[i] = i == 0 ? 0 : ((i % 2 == 1) ? i + 1 : i - 1);
  }
  return L;
}

// ---------------------------------------------------------------- device arena
struct Arena {
  std::vector<void*> ptrs;
  ~Arena() { for (void* p : ptrs) cudaFree(p); }
  void* alloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
};

// ---------------------------------------------------------------- step DAG
struct TermSpec {       // host-side description of a term, resolved to MpsRef at build time
  int kind = T_PLAIN;
  int x = -1, y = -1;   // node ids
  double coef = 1.0;
  int coef_slot = -1;
  int axis = 0, offset = 0, cyclic = 1;
  int mask_id = -1;
};

struct JobSpec {
  int kind;             // 0 rounding, 1 fit, 2 rho0 scalar, 3 zip-up pass
  int out;              // node id
  std::vector<TermSpec> terms;
  int b = -1, c = -1;   // fit factors
  int level = 0;
};

}  // namespace tn

using namespace tn;

struct tnlbm_sim {
  tnlbm_config cfg{};
  int n = 0, L = 0, N = 0, prec = 0;
  size_t esz = 8;
  LatticeDef lat{};
  Arena arena;
  cudaStream_t s0 = nullptr, s1 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // nodes
  std::vector<MpsRef> nodes;
  std::vector<int> node_level;
  int scal_node = -1;
  std::vector<int> f_state, f_next;
  int mask_node = -1;
  int rho_node = -1;
  double n_fluid = 0.0;
  // masks (rank-1 wall planes) [id][TN_MAXL][2]
  std::vector<double> mask_vecs;
  void* d_masks = nullptr;
  double* d_scal = nullptr;
  int* d_status = nullptr;
  // jobs per level
  std::vector<JobSpec> specs;
  struct Level {
    std::vector<RoundJob> rj;
    std::vector<FitJob> fj;
    std::vector<ZipJob> zj;
    RoundJob* d_rj = nullptr;
    FitJob* d_fj = nullptr;
    ZipJob* d_zj = nullptr;
    bool has_rho0 = false;
    int cluster = 1;               // CTAs per rounding job of this level
  };
  std::vector<Level> levels;
  MpsRef* d_rho_ref = nullptr;
  MpsRef* d_copy_src = nullptr;
  MpsRef* d_copy_dst = nullptr;
  double* d_mass = nullptr;      // [Q] per-population masses (mass correction)
  double* d_mass0 = nullptr;     // initial total mass
  double* d_discard = nullptr;   // squared discarded tails of all roundings so far
  int launches_per_step = 0;
  int64_t steps = 0;
  int pending_status = 0;
  // learned rounding (rank model + randomized truncation); off until configured
  int learn_mode = 0;            // 0 off, 1 log spectra, 2 predict ranks
  LearnCtx h_learn{};
  LearnCtx* d_learn = nullptr;
  JobLog* d_logs = nullptr;
  int n_logs = 0;
  int* d_step = nullptr;
  int* d_lcount = nullptr;       // [0] accepted, [1] fell back, [2] full SVDs, [3] dataset rows
  void* d_omega = nullptr;
  size_t omega_bytes = 0;
  float* d_dataset = nullptr;
  int dataset_cap = 0;
  __half* d_mlp = nullptr;
  bool mlp_set = false;
};

namespace tn {

static int new_node(tnlbm_sim* s, int cap, int level) {
  MpsRef m{};
  m.cap = cap;
  m.base = s->arena.alloc(mps_size(s->L, cap) * s->esz);
  m.ranks = (int*)s->arena.alloc((s->L + 1) * sizeof(int));
  if (!m.base || !m.ranks) return -1;
  std::vector<int> ones(s->L + 1, 1);
  cudaMemcpy(m.ranks, ones.data(), ones.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemset(m.base, 0, mps_size(s->L, cap) * s->esz);
  s->nodes.push_back(m);
  s->node_level.push_back(level);
  return (int)s->nodes.size() - 1;
}

struct Builder {
  tnlbm_sim* s;
  bool oom = false;
  int chi() const { return s->cfg.chi_max; }

  int level_of_terms(const std::vector<TermSpec>& ts) {
    int lv = 0;
    for (const TermSpec& t : ts) {
      if (t.x >= 0) lv = std::max(lv, s->node_level[t.x]);
      if (t.y >= 0) lv = std::max(lv, s->node_level[t.y]);
      if (t.coef_slot >= 0) lv = std::max(lv, s->node_level[s->scal_node]);
    }
    return lv + 1;
  }
  int R(const std::vector<TermSpec>& ts) {
    int lv = level_of_terms(ts);
    int out = new_node(s, chi(), lv);
    if (out < 0) { oom = true; return -1; }
    JobSpec j;
    j.kind = 0; j.out = out; j.terms = ts; j.level = lv;
    s->specs.push_back(j);
    return out;
  }
  int H(int b, int c) {
    if (s->cfg.hadamard == TNLBM_HADAMARD_EXACT) {
      TermSpec t; t.kind = T_KRON; t.x = b; t.y = c;
      return R({t});
    }
    if (s->cfg.hadamard == TNLBM_HADAMARD_ZIPUP) {      // zip-up pass, then a rounding
      int lv = std::max(s->node_level[b], s->node_level[c]) + 1;
      int z = new_node(s, chi(), lv);
      if (z < 0) { oom = true; return -1; }
      JobSpec j;
      j.kind = 3; j.out = z; j.b = b; j.c = c; j.level = lv;
      s->specs.push_back(j);
      return R({P(z, 1.0)});
    }
    int lv = std::max(s->node_level[b], s->node_level[c]) + 1;
    int out = new_node(s, s->nodes[b].cap, lv);
    if (out < 0) { oom = true; return -1; }
    JobSpec j;
    j.kind = 1; j.out = out; j.b = b; j.c = c; j.level = lv;
    s->specs.push_back(j);
    return out;
  }
  static TermSpec P(int x, double c, int slot = -1) {
    TermSpec t; t.kind = T_PLAIN; t.x = x; t.coef = c; t.coef_slot = slot; return t;
  }
  static TermSpec ONE(double c, int slot = -1) {
    TermSpec t; t.kind = T_ONES; t.coef = c; t.coef_slot = slot; return t;
  }
  TermSpec SH(int x, int axis, int cd) {
    TermSpec t; t.kind = T_SHIFT; t.x = x; t.axis = axis; t.offset = -cd;
    t.cyclic = s->cfg.periodic[axis] ? 1 : 0;
    return t;
  }
  int mask_plane_product(const std::vector<int>& axes, const int* c) {
    // rank-1 product of plane indicators x_d = 0 (c_d > 0) or N-1 (c_d < 0)
    int id = (int)(s->mask_vecs.size() / (TN_MAXL * 2));
    s->mask_vecs.resize(s->mask_vecs.size() + TN_MAXL * 2, 1.0);
    double* v = &s->mask_vecs[(size_t)id * TN_MAXL * 2];
    for (int k = 0; k < s->L; ++k) {
      int d = k % 3;
      if (std::find(axes.begin(), axes.end(), d) != axes.end()) {
        v[2 * k + 0] = c[d] > 0 ? 1.0 : 0.0;
        v[2 * k + 1] = c[d] > 0 ? 0.0 : 1.0;
      }
    }
    return id;
  }

  int tree_sum(std::vector<TermSpec> items) {
    if (s->cfg.block_sums && items.size() > 1) return R(items);   // one rounding of the block sum
    while (items.size() > 1) {
      std::vector<TermSpec> nxt;
      for (size_t p = 0; p + 1 < items.size(); p += 2) nxt.push_back(P(R({items[p], items[p + 1]}), 1.0));
      if (items.size() % 2 == 1) nxt.push_back(items.back());
      items = nxt;
    }
    if (items[0].coef == 1.0) return items[0].x;
    return R({items[0]});
  }

  void build_step() {
    tnlbm_sim& S = *s;
    const LatticeDef& lat = S.lat;
    const int Q = lat.Q;
    const double tau = S.cfg.tau, omega = 1.0 / tau;
    // a1 moments
    std::vector<TermSpec> it;
    for (int i = 0; i < Q; ++i) it.push_back(P(S.f_state[i], 1.0));
    int rho = tree_sum(it);
    S.rho_node = rho;
    int j[3];
    for (int d = 0; d < 3; ++d) {
      std::vector<TermSpec> v;
      for (int i = 0; i < Q; ++i)
        if (lat.c[i][d] != 0) v.push_back(P(S.f_state[i], (double)lat.c[i][d]));
      j[d] = tree_sum(v);
    }
    // a2 rho_0 (a scalar pseudo-node)
    S.scal_node = new_node(s, 1, S.node_level[rho] + 1);
    {
      JobSpec js; js.kind = 2; js.out = S.scal_node; js.b = rho; js.level = S.node_level[S.scal_node];
      S.specs.push_back(js);
    }
    // a3
    int drho = R({P(rho, 1.0), ONE(1.0, SC_NEG_RHO0)});
    int sq = H(drho, drho);
    int inv = R({ONE(1.0, SC_INV1), P(drho, 1.0, SC_INV2), P(sq, 1.0, SC_INV3)});
    // a4
    int Jt[3];
    for (int d = 0; d < 3; ++d) {
      const double F = S.cfg.force[d];
      if (F == 0.0) { Jt[d] = j[d]; continue; }
      std::vector<TermSpec> ts = {P(j[d], 1.0), ONE(tau * F)};
      if (S.mask_node >= 0) ts.push_back(P(S.mask_node, -tau * F));
      Jt[d] = R(ts);
    }
    int u[3];
    for (int d = 0; d < 3; ++d) u[d] = H(Jt[d], inv);
    // a5
    int Pm[3][3];
    for (int d = 0; d < 3; ++d)
      for (int e = d; e < 3; ++e) Pm[d][e] = H(Jt[d], u[e]);
    // a6
    int E0 = rho;
    for (int d = 0; d < 3; ++d) E0 = R({P(E0, 1.0), P(Pm[d][d], -1.5)});
    std::map<std::vector<std::pair<int, double>>, int> qcache;   // key: (de code, kappa)
    std::map<std::vector<std::pair<int, double>>, int> vcache;
    auto qchain = [&](auto&& self, const std::vector<std::pair<int, double>>& key) -> int {
      if (key.empty()) return E0;
      auto itq = qcache.find(key);
      if (itq != qcache.end()) return itq->second;
      std::vector<std::pair<int, double>> pre(key.begin(), key.end() - 1);
      int prev = self(self, pre);
      int de = key.back().first;
      int out = R({P(prev, 1.0), P(Pm[de / 3][de % 3], key.back().second)});
      qcache[key] = out;
      return out;
    };
    // returns term (coef, node) for a first-order key
    auto vchain = [&](auto&& self, const std::vector<std::pair<int, double>>& key) -> TermSpec {
      if (key.size() == 1) return P(Jt[key[0].first], key[0].second);
      auto itv = vcache.find(key);
      if (itv != vcache.end()) return P(itv->second, 1.0);
      std::vector<std::pair<int, double>> pre(key.begin(), key.end() - 1);
      TermSpec prev = self(self, pre);
      int out = R({prev, P(Jt[key.back().first], key.back().second)});
      vcache[key] = out;
      return P(out, 1.0);
    };
    std::vector<int> fstar(Q);
    for (int i = 0; i < Q; ++i) {
      const int* c = lat.c[i];
      std::vector<std::pair<int, double>> qk;
      for (int d = 0; d < 3; ++d)
        if (c[d] != 0) qk.push_back({d * 3 + d, 4.5 * c[d] * c[d]});
      const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
      for (auto& pr : pairs)
        if (c[pr[0]] != 0 && c[pr[1]] != 0) qk.push_back({pr[0] * 3 + pr[1], 9.0 * c[pr[0]] * c[pr[1]]});
      int Qi = qchain(qchain, qk);
      std::vector<std::pair<int, double>> first;
      for (int d = 0; d < 3; ++d)
        if (c[d] != 0) first.push_back({d, 3.0 * c[d]});
      int Y;
      if (!first.empty()) {
        const double sigma = first[0].second > 0 ? 1.0 : -1.0;
        for (auto& p : first) p.second *= sigma;
        TermSpec v = vchain(vchain, first);
        v.coef *= sigma;
        Y = R({P(Qi, 1.0), v});
      } else {
        Y = Qi;
      }
      fstar[i] = R({P(S.f_state[i], 1.0 - omega), P(Y, omega * lat.w[i])});
    }
    // a7 streaming
    bool use_faces = false;
    for (int f6 = 0; f6 < 6; ++f6) use_faces = use_faces || S.cfg.face_kind[f6] != TNLBM_FACE_WALL;
    int ones_node = -1;
    if (use_faces) {
      // the all-ones MPS (rank 1), operand of the masked constant terms
      ones_node = new_node(s, 1, 0);
      if (ones_node < 0) { oom = true; return; }
      const size_t ne = mps_size(S.L, 1);
      if (S.prec == TNLBM_FP64) {
        std::vector<double> h(ne, 1.0);
        cudaMemcpy(S.nodes[ones_node].base, h.data(), ne * sizeof(double), cudaMemcpyHostToDevice);
      } else {
        std::vector<float> h(ne, 1.0f);
        cudaMemcpy(S.nodes[ones_node].base, h.data(), ne * sizeof(float), cudaMemcpyHostToDevice);
      }
    }
    std::vector<int> fs(Q);
    for (int i = 0; i < Q; ++i) {
      const int* c = lat.c[i];
      std::vector<int> axes;
      for (int d = 0; d < 3; ++d) if (c[d] != 0) axes.push_back(d);
      int x = fstar[i];
      std::vector<int> W;
      for (int d : axes) if (!S.cfg.periodic[d]) W.push_back(d);
      for (size_t t = 0; t < axes.size(); ++t) {
        std::vector<TermSpec> ts = {SH(x, axes[t], c[axes[t]])};
        if (t + 1 == axes.size() && !use_faces) {
          for (int bits = 1; bits < (1 << W.size()); ++bits) {
            std::vector<int> sub;
            for (size_t q = 0; q < W.size(); ++q) if (bits >> q & 1) sub.push_back(W[q]);
            TermSpec m; m.kind = T_MASK1; m.x = fstar[lat.opp[i]];
            m.coef = (sub.size() % 2 == 1) ? 1.0 : -1.0;
            m.mask_id = mask_plane_product(sub, c);
            ts.push_back(m);
          }
        } else if (t + 1 == axes.size()) {
          // per-face boundary functions: the cells entered through wall axis
          // W[wi] and none of lower index, plane_d prod (1 - plane_d') expanded
          const double wi_ = lat.w[i];
          for (size_t wi = 0; wi < W.size(); ++wi) {
            const int d = W[wi];
            const int face = 2 * d + (c[d] > 0 ? 0 : 1);
            const int kind = S.cfg.face_kind[face];
            for (int bits = 0; bits < (1 << wi); ++bits) {
              std::vector<int> axset = {d};
              int cnt = 0;
              for (size_t q = 0; q < wi; ++q)
                if (bits >> q & 1) { axset.push_back(W[q]); ++cnt; }
              const double sgn = (cnt % 2) ? -1.0 : 1.0;
              const int mid = mask_plane_product(axset, c);
              auto MK = [&](int node, double coef, int slot) {
                TermSpec m; m.kind = T_MASK1; m.x = node; m.coef = coef; m.coef_slot = slot; m.mask_id = mid;
                return m;
              };
              if (kind == TNLBM_FACE_WALL) {
                ts.push_back(MK(fstar[lat.opp[i]], sgn, -1));
              } else if (kind == TNLBM_FACE_VELOCITY) {
                ts.push_back(MK(fstar[lat.opp[i]], sgn, -1));
                for (int e = 0; e < 3; ++e)          // 2 w_i c_ie (rho_0 u_b,e) / c_s^2
                  if (c[e] != 0) ts.push_back(MK(ones_node, sgn * 6.0 * wi_ * c[e], SC_UB + 3 * face + e));
              } else {
                const double rb = S.cfg.face_rho[face];
                ts.push_back(MK(fstar[lat.opp[i]], -sgn, -1));
                ts.push_back(MK(ones_node, sgn * 2.0 * wi_ * rb, -1));
                for (int d1 = 0; d1 < 3; ++d1)
                  for (int e1 = d1; e1 < 3; ++e1) {
                    const double kap = d1 == e1 ? 4.5 * c[d1] * c[d1] - 1.5 : 9.0 * c[d1] * c[e1];
                    if (kap != 0.0) ts.push_back(MK(Pm[d1][e1], sgn * 2.0 * wi_ * rb * kap, SC_INV1));
                  }
              }
            }
          }
        }
        x = R(ts);
      }
      fs[i] = x;
    }
    std::vector<int> out = fs;
    if (S.mask_node >= 0) {
      // a8 objects
      std::vector<int> g(Q, -1);
      for (int i = 1; i < Q; ++i) g[i] = H(fs[i], S.mask_node);
      for (int i = 1; i < Q; ++i) {
        const int* c = lat.c[i];
        int h = g[lat.opp[i]];
        for (int d = 0; d < 3; ++d) if (c[d] != 0) h = R({SH(h, d, c[d])});
        int t = R({P(fs[i], 1.0), P(g[i], -1.0)});
        out[i] = R({P(t, 1.0), P(h, 1.0)});
      }
    }
    S.f_next = out;
  }
};

// Options every rounding job of a simulation carries.
static void set_round_options(const tnlbm_sim* s, RoundJob& rj) {
  rj.svd64 = prec_svd64(s->prec) ? 1 : 0;
  rj.max_sweeps = s->cfg.jacobi_max_sweeps;
  rj.wait_ns = s->cfg.wait_limit_ns;
}

// CTAs per rounding job for a launch of njobs jobs of a simulation: clusters
// share the FP64 centre SVDs (TNLBM_MIXED, TNLBM_BF16 and TNLBM_FP64); FP32 jobs run alone.
template <typename T>
static int sim_cluster(const tnlbm_sim* s, int njobs) {
  if (!prec_svd64(s->prec) && s->prec != TNLBM_FP64) return 1;
  const int cap = s->cfg.max_cluster > 0 ? s->cfg.max_cluster : 16;
  return cap <= 1 ? 1 : round_cluster_size<T>(njobs, cap);
}

template <typename T>
static int upload_levels(tnlbm_sim* s) {
  // group specs by level, materialise RoundJobs / FitJobs with scratch shared across levels
  int maxlv = 0;
  for (auto& j : s->specs) maxlv = std::max(maxlv, j.level);
  s->levels.assign(maxlv + 1, tnlbm_sim::Level{});
  size_t round_scr = 0, fit_scr = 0;
  std::vector<size_t> lvl_round(maxlv + 1, 0), lvl_fit(maxlv + 1, 0);
  for (auto& js : s->specs) {
    tnlbm_sim::Level& lv = s->levels[js.level];
    if (js.kind == 2) { lv.has_rho0 = true; continue; }
    if (js.kind == 0) {
      RoundJob rj{};
      rj.nterms = (int)js.terms.size();
      if (rj.nterms > TN_MAXT) { set_error("too many terms in a rounding job"); return TNLBM_E_ARG; }
      rj.chi = s->cfg.chi_max;
      rj.eps = s->cfg.eps;
      for (int t = 0; t < rj.nterms; ++t) {
        const TermSpec& ts = js.terms[t];
        Term& tm = rj.t[t];
        tm.kind = ts.kind; tm.axis = ts.axis; tm.offset = ts.offset; tm.cyclic = ts.cyclic;
        tm.coef = ts.coef; tm.coef_slot = ts.coef_slot; tm.mask_id = ts.mask_id;
        if (ts.x >= 0) tm.x = s->nodes[ts.x];
        if (ts.y >= 0) tm.y = s->nodes[ts.y];
      }
      rj.dst = s->nodes[js.out];
      rj.discard = s->d_discard;
      set_round_options(s, rj);
      plan_round_job(rj, s->L, s->n, sizeof(T));
      lvl_round[js.level] += rj.lay.total;
      lv.rj.push_back(rj);
    } else if (js.kind == 3) {
      ZipJob zj{};
      zj.B = s->nodes[js.b];
      zj.C = s->nodes[js.c];
      zj.Z = s->nodes[js.out];
      zj.chi = s->cfg.chi_max;
      zj.eps = s->cfg.eps;
      lvl_fit[js.level] += zip_scratch_elems(s->L, zj.B.cap, zj.C.cap, zj.Z.cap, sizeof(T));
      lv.zj.push_back(zj);
    } else {
      FitJob fj{};
      fj.A = s->nodes[js.out];
      fj.B = s->nodes[js.b];
      fj.C = s->nodes[js.c];
      size_t env, xs, ys, ab, q;
      plan_fit_job(fj, s->L, &env, &xs, &ys, &ab, &q);
      fj.env_stride = env;
      fj.qscr_stride = q;
      lvl_fit[js.level] += 2 * (s->L + 1) * env + xs + ys + ab + 4 * q;
      lv.fj.push_back(fj);
    }
  }
  for (int l = 0; l <= maxlv; ++l) {
    round_scr = std::max(round_scr, lvl_round[l]);
    fit_scr = std::max(fit_scr, lvl_fit[l]);
  }
  T* rbase = (T*)s->arena.alloc(round_scr * sizeof(T));
  T* fbase = (T*)s->arena.alloc(fit_scr * sizeof(T));
  if (!rbase || !fbase) { set_error("out of device memory for scratch"); return TNLBM_E_OOM; }
  for (auto& lv : s->levels) {
    size_t o = 0;
    for (auto& rj : lv.rj) { rj.scratch = rbase + o; o += rj.lay.total; }
    o = 0;
    for (auto& fj : lv.fj) {
      size_t env, xs, ys, ab, q;
      plan_fit_job(fj, s->L, &env, &xs, &ys, &ab, &q);
      fj.env_l = fbase + o; o += (s->L + 1) * env;
      fj.env_r = fbase + o; o += (s->L + 1) * env;
      fj.x = fbase + o; o += xs;
      fj.y = fbase + o; o += ys;
      fj.abuf = fbase + o; o += ab;
      fj.qscr = fbase + o; o += 4 * q;
    }
    for (auto& zj : lv.zj) {
      zj.scratch = fbase + o;
      o += zip_scratch_elems(s->L, zj.B.cap, zj.C.cap, zj.Z.cap, sizeof(T));
    }
    if (!lv.zj.empty()) {
      lv.d_zj = (ZipJob*)s->arena.alloc(lv.zj.size() * sizeof(ZipJob));
      if (!lv.d_zj) return TNLBM_E_OOM;
      cudaMemcpy(lv.d_zj, lv.zj.data(), lv.zj.size() * sizeof(ZipJob), cudaMemcpyHostToDevice);
    }
    if (!lv.rj.empty()) {
      lv.d_rj = (RoundJob*)s->arena.alloc(lv.rj.size() * sizeof(RoundJob));
      if (!lv.d_rj) return TNLBM_E_OOM;
      cudaMemcpy(lv.d_rj, lv.rj.data(), lv.rj.size() * sizeof(RoundJob), cudaMemcpyHostToDevice);
      lv.cluster = sim_cluster<T>(s, (int)lv.rj.size());
    }
    if (!lv.fj.empty()) {
      lv.d_fj = (FitJob*)s->arena.alloc(lv.fj.size() * sizeof(FitJob));
      if (!lv.d_fj) return TNLBM_E_OOM;
      cudaMemcpy(lv.d_fj, lv.fj.data(), lv.fj.size() * sizeof(FitJob), cudaMemcpyHostToDevice);
    }
  }
  return 0;
}

template <typename T>
static int enqueue_step(tnlbm_sim* s, int* launches, Prof* prof = nullptr) {
  int n = 0;
  double* ctr = prof ? prof->d_ctr : nullptr;
  for (auto& lv : s->levels) {
    if (lv.has_rho0) {
      launch_rho0<T>(s->d_rho_ref, s->L, s->n_fluid, s->d_scal, s->s0);
      if (prof) prof->mark(C_RHO0);
      ++n;
    }
    const bool side = !lv.fj.empty() || !lv.zj.empty();
    const bool both = !prof && !lv.rj.empty() && side;   // profiled runs stay serial
    if (both) {
      cudaEventRecord(s->ev_fork, s->s0);
      cudaStreamWaitEvent(s->s1, s->ev_fork, 0);
    }
    if (!lv.fj.empty())
      n += run_fit<T>(lv.d_fj, lv.fj, s->L, s->cfg.sweeps, s->d_status, both ? s->s1 : s->s0, prof,
                      prec_tc(s->prec));
    if (!lv.zj.empty()) {
      n += run_zipup<T>(lv.d_zj, (int)lv.zj.size(), s->L, s->d_status, both ? s->s1 : s->s0, ctr);
      if (prof) prof->mark(C_ZIPUP);
    }
    if (!lv.rj.empty()) {
      launch_round<T>(lv.d_rj, (int)lv.rj.size(), s->L, s->n, (const T*)s->d_masks, s->d_scal,
                      s->d_status, s->s0, ctr, s->learn_mode ? s->d_learn : nullptr, lv.cluster);
      if (prof) prof->mark(C_ROUND);
      ++n;
    }
    if (both) {
      cudaEventRecord(s->ev_join, s->s1);
      cudaStreamWaitEvent(s->s0, s->ev_join, 0);
    }
  }
  if (s->cfg.conserve_mass) {
    launch_mass_fix<T>(s->d_copy_src, s->lat.Q, s->L, s->d_mass, s->d_mass0, s->s0);
    if (prof) prof->mark(C_COPY);
    n += 2;
  }
  launch_copy<T>(s->d_copy_src, s->d_copy_dst, s->lat.Q, s->L, s->s0);
  if (prof) prof->mark(C_COPY);
  ++n;
  if (s->learn_mode) {
    launch_learn_tick(s->d_step, s->s0);
    ++n;
  }
  *launches = n;
  return 0;
}

// (re)capture one step as a graph
template <typename T>
static int capture_graph(tnlbm_sim* s) {
  TN_CUDA(cudaStreamSynchronize(s->s0));
  if (s->gexec) { cudaGraphExecDestroy(s->gexec); s->gexec = nullptr; }
  if (s->graph) { cudaGraphDestroy(s->graph); s->graph = nullptr; }
  TN_CUDA(cudaStreamBeginCapture(s->s0, cudaStreamCaptureModeThreadLocal));
  int launches = 0;
  enqueue_step<T>(s, &launches);
  TN_CUDA(cudaStreamEndCapture(s->s0, &s->graph));
  TN_CUDA(cudaGraphInstantiate(&s->gexec, s->graph, 0));
  s->launches_per_step = launches;
  return 0;
}

// ------------------------------------------------------------ cluster tuning
// Cluster sizes the tuner times for a rounding launch (largest first), besides
// the size the level already has.
static const int TUNE_P[] = {16, 8, 4, 2, 1};

// Times run(P) -- one rounding launch of a level with clusters of P CTAs, on
// stream st -- at the current size `cur`, then at the sizes of TUNE_P, then
// at 3/4 and 3/2 of the fastest of those, among the sizes that fit (P <= cap
// and resident on this device); each time is the minimum of `reps` launches.
// Below cur, smaller sizes of TUNE_P are skipped once one is 1.5x slower than
// the best so far: with more jobs than fit at once, large clusters run in
// waves, while small ones spread each FP64 SVD over fewer SMs, so the time
// falls and then rises as P shrinks.  ms[P] gets the time of size P (-1 where
// not timed); *best the fastest, where cur stays unless another size is 2 %
// faster.  Every launch writes the level's outputs again, from the same
// inputs.
template <typename T, typename F>
static int tune_launch(F&& run, int cap, int reps, int cur, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                       double* ms, int* best) {
  double t[TNLBM_CLUSTER_MAX + 1];
  for (int P = 0; P <= TNLBM_CLUSTER_MAX; ++P) t[P] = -1.0;
  std::vector<int> cand;                    // the current size first, then the others from 16 down
  if (cur >= 1 && cur <= TNLBM_CLUSTER_MAX && round_cluster_resident<T>(cur) >= 1) cand.push_back(cur);
  for (int P : TUNE_P)
    if (P != cur && P <= cap && round_cluster_resident<T>(P) >= 1) cand.push_back(P);
  auto time_at = [&](int P, double* out) -> int {
    double tm = 1e300;
    for (int r = 0; r < std::max(reps, 1); ++r) {
      TN_CUDA(cudaEventRecord(e0, st));
      run(P);
      TN_CUDA(cudaGetLastError());
      TN_CUDA(cudaEventRecord(e1, st));
      TN_CUDA(cudaEventSynchronize(e1));
      float f = 0.f;
      TN_CUDA(cudaEventElapsedTime(&f, e0, e1));
      tm = std::min(tm, (double)f);
    }
    *out = tm;
    return 0;
  };
  int pb = -1;
  for (int P : cand) {
    const int rc = time_at(P, &t[P]);
    if (rc) return rc;
    if (pb < 0 || t[P] < t[pb]) pb = P;
    else if (P < cur || cur < 1) {
      if (t[P] > 1.5 * t[pb]) break;
    }
  }
  if (pb < 0) { set_error("no cluster size of the rounding kernel fits on this device"); return TNLBM_E_CUDA; }
  // then the sizes halfway to the best one's neighbours (3 and 6 around 4,
  // 6 and 12 around 8, ...): the number of waves moves in steps of whole
  // waves, so the optimum need not be a power of two
  const int best2 = pb;
  for (int P : {best2 * 3 / 4, best2 * 3 / 2}) {
    if (P < 1 || P > cap || P > TNLBM_CLUSTER_MAX || t[P] >= 0.0) continue;
    if (round_cluster_resident<T>(P) < 1) continue;
    const int rc = time_at(P, &t[P]);
    if (rc) return rc;
    if (t[P] < t[pb]) pb = P;
  }
  if (cur >= 1 && cur <= TNLBM_CLUSTER_MAX && t[cur] >= 0.0 && t[cur] <= 1.02 * t[pb]) pb = cur;
  if (ms)
    for (int P = 0; P <= TNLBM_CLUSTER_MAX; ++P) ms[P] = t[P];
  *best = pb;
  return 0;
}

// Whether the rounding jobs of a precision run as clusters: the CTAs of a
// cluster share the FP64 centre SVDs, so FP32 and TF32 jobs run one CTA each.
static bool clusters_apply(int prec) { return prec_svd64(prec) || prec == TNLBM_FP64; }

// Checks a cluster size given for a level of njobs rounding jobs.
template <typename T>
static int check_cluster(int prec, int P) {
  if (P < 1 || P > TNLBM_CLUSTER_MAX) { set_error("cluster sizes are 1..16"); return TNLBM_E_ARG; }
  if (P > 1 && !clusters_apply(prec)) {
    set_error("FP32 and TF32 rounding jobs run one CTA each (cluster size 1)");
    return TNLBM_E_ARG;
  }
  if (round_cluster_resident<T>(P) < 1) {
    set_error("clusters of " + std::to_string(P) + " CTAs of the rounding kernel do not fit on this device");
    return TNLBM_E_ARG;
  }
  return 0;
}

// Runs one step of a simulation eagerly on s0, level by level, timing each
// rounding launch at every candidate cluster size and keeping the fastest;
// the final copy into the populations (and the mass correction before it) is
// left out, so the state, the step count and the discarded-weight total are
// as before.  ms: [levels][17] times (may be NULL).  Re-captures the graph.
template <typename T>
static int tune_sim(tnlbm_sim* s, int reps, double* ms, int ms_cap) {
  if (s->learn_mode) { set_error("tune the cluster sizes before configuring the learned rounding"); return TNLBM_E_ARG; }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  double disc = 0.0;
  TN_CUDA(cudaMemcpy(&disc, s->d_discard, sizeof(double), cudaMemcpyDeviceToHost));
  const int cap = s->cfg.max_cluster > 0 ? std::min(s->cfg.max_cluster, (int)TNLBM_CLUSTER_MAX) : TNLBM_CLUSTER_MAX;
  const bool tune = clusters_apply(s->prec) && cap > 1;
  std::vector<int> old;
  for (auto& lv : s->levels) old.push_back(lv.cluster);
  std::vector<double> t((size_t)s->levels.size() * (TNLBM_CLUSTER_MAX + 1), -1.0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TN_CUDA(cudaEventCreate(&e0));
  TN_CUDA(cudaEventCreate(&e1));
  int rc = 0;
  for (size_t l = 0; l < s->levels.size() && !rc; ++l) {
    auto& lv = s->levels[l];
    if (lv.has_rho0) launch_rho0<T>(s->d_rho_ref, s->L, s->n_fluid, s->d_scal, s->s0);
    if (!lv.fj.empty())
      run_fit<T>(lv.d_fj, lv.fj, s->L, s->cfg.sweeps, s->d_status, s->s0, nullptr, prec_tc(s->prec));
    if (!lv.zj.empty()) run_zipup<T>(lv.d_zj, (int)lv.zj.size(), s->L, s->d_status, s->s0, nullptr);
    if (lv.rj.empty()) continue;
    auto run = [&](int P) {
      launch_round<T>(lv.d_rj, (int)lv.rj.size(), s->L, s->n, (const T*)s->d_masks, s->d_scal, s->d_status,
                      s->s0, nullptr, nullptr, P);
    };
    if (tune) {
      int best = lv.cluster;
      rc = tune_launch<T>(run, cap, reps, lv.cluster, s->s0, e0, e1, t.data() + l * (TNLBM_CLUSTER_MAX + 1), &best);
      if (!rc) lv.cluster = best;
    } else {
      run(lv.cluster);
    }
  }
  cudaStreamSynchronize(s->s0);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TN_CUDA(cudaMemcpy(s->d_discard, &disc, sizeof(double), cudaMemcpyHostToDevice));
  int st[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpy(st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (!rc && st[0]) {
    rc = status_to_code(st);
    TN_CUDA(cudaMemset(s->d_status, 0, STATUS_INTS * sizeof(int)));
  }
  if (rc)
    for (size_t l = 0; l < s->levels.size(); ++l) s->levels[l].cluster = old[l];
  else if (ms)
    std::copy(t.begin(), t.begin() + std::min<size_t>(t.size(), std::max(ms_cap, 0)), ms);
  const int rc2 = capture_graph<T>(s);
  return rc ? rc : rc2;
}

// Switch the learned rounding of a simulation (see tnlbm_learn_configure).
template <typename T>
static int learn_configure_impl(tnlbm_sim* s, int mode, const double* omega, int rows, int ld,
                                int oversample, int power, double eta, double floor_rel, int dataset_cap) {
  if (!s->d_learn) {
    int nj = 0;
    for (auto& lv : s->levels) nj += (int)lv.rj.size();
    s->n_logs = nj;
    s->d_learn = (LearnCtx*)s->arena.alloc(sizeof(LearnCtx));
    s->d_logs = (JobLog*)s->arena.alloc(std::max(nj, 1) * sizeof(JobLog));
    s->d_step = (int*)s->arena.alloc(sizeof(int));
    s->d_lcount = (int*)s->arena.alloc(4 * sizeof(int));
    s->d_mlp = (__half*)s->arena.alloc(MLP_NPARAM * sizeof(__half));
    if (!s->d_learn || !s->d_logs || !s->d_step || !s->d_lcount || !s->d_mlp) {
      set_error("out of device memory for the learned rounding");
      return TNLBM_E_OOM;
    }
    TN_CUDA(cudaMemset(s->d_mlp, 0, MLP_NPARAM * sizeof(__half)));
  }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  if (mode > 0) {
    const size_t ob = (size_t)rows * ld * sizeof(T);
    if (ob > s->omega_bytes) {
      s->d_omega = s->arena.alloc(ob);
      if (!s->d_omega) { set_error("out of device memory for omega"); return TNLBM_E_OOM; }
      s->omega_bytes = ob;
    }
    std::vector<T> ho((size_t)rows * ld);
    for (size_t i = 0; i < ho.size(); ++i) ho[i] = (T)omega[i];
    TN_CUDA(cudaMemcpy(s->d_omega, ho.data(), ob, cudaMemcpyHostToDevice));
    if (dataset_cap > s->dataset_cap) {
      s->d_dataset = (float*)s->arena.alloc((size_t)dataset_cap * (MLP_IN + 1) * sizeof(float));
      if (!s->d_dataset) { set_error("out of device memory for the spectrum log"); return TNLBM_E_OOM; }
      s->dataset_cap = dataset_cap;
    }
  }
  const int step = (int)std::min<int64_t>(s->steps, 1 << 30);
  TN_CUDA(cudaMemcpy(s->d_step, &step, sizeof(int), cudaMemcpyHostToDevice));
  TN_CUDA(cudaMemset(s->d_lcount, 0, 4 * sizeof(int)));
  TN_CUDA(cudaMemset(s->d_logs, 0, std::max(s->n_logs, 1) * sizeof(JobLog)));
  LearnCtx& h = s->h_learn;
  h = LearnCtx{};
  h.omega = s->d_omega;
  h.omega_rows = rows;
  h.omega_ld = ld;
  h.oversample = oversample;
  h.power = power;
  h.eta = (float)eta;
  h.floor_rel = (float)floor_rel;
  h.mlp = s->d_mlp;
  h.step = s->d_step;
  h.dataset = dataset_cap > 0 ? s->d_dataset : nullptr;
  h.dataset_count = s->d_lcount + 3;
  h.dataset_cap = dataset_cap;
  h.counters = s->d_lcount;
  TN_CUDA(cudaMemcpy(s->d_learn, &h, sizeof(LearnCtx), cudaMemcpyHostToDevice));
  int idx = 0;
  for (auto& lv : s->levels) {
    for (auto& rj : lv.rj) {
      rj.rsvd_mode = (mode >= 2) ? mode : 0;
      rj.log = mode > 0 ? s->d_logs + idx : nullptr;
      ++idx;
    }
    if (!lv.rj.empty())
      TN_CUDA(cudaMemcpy(lv.d_rj, lv.rj.data(), lv.rj.size() * sizeof(RoundJob), cudaMemcpyHostToDevice));
  }
  s->learn_mode = mode;
  return capture_graph<T>(s);
}

// one-off rounding jobs (initial states): terms over nodes
template <typename T>
static int run_round_now(tnlbm_sim* s, std::vector<RoundJob>& jobs) {
  if (jobs.empty()) return 0;
  size_t tot = 0;
  for (auto& j : jobs) { set_round_options(s, j); plan_round_job(j, s->L, s->n, sizeof(T)); tot += j.lay.total; }
  T* scr = nullptr;
  RoundJob* dj = nullptr;
  if (cudaMalloc(&scr, std::max<size_t>(tot, 1) * sizeof(T)) != cudaSuccess) return TNLBM_E_OOM;
  size_t o = 0;
  for (auto& j : jobs) { j.scratch = scr + o; o += j.lay.total; }
  if (cudaMalloc(&dj, jobs.size() * sizeof(RoundJob)) != cudaSuccess) { cudaFree(scr); return TNLBM_E_OOM; }
  cudaMemcpy(dj, jobs.data(), jobs.size() * sizeof(RoundJob), cudaMemcpyHostToDevice);
  launch_round<T>(dj, (int)jobs.size(), s->L, s->n, (const T*)s->d_masks, s->d_scal, s->d_status, s->s0,
                  nullptr, nullptr, sim_cluster<T>(s, (int)jobs.size()));
  cudaError_t e = cudaStreamSynchronize(s->s0);
  cudaFree(scr);
  cudaFree(dj);
  if (e != cudaSuccess) return cuda_fail(e, "initial rounding");
  return 0;
}

static void mode_cores(int n_bits, const double* row, std::vector<std::vector<double>>& cores) {
  // exact rank-2 MPS of cos(2 pi k.x / N + phase): each site rotates the running
  // (cos, sin) pair by its bit's phase
  const int L = 3 * n_bits;
  const double N = (double)(1 << n_bits);
  cores.assign(L, {});
  for (int s = 0; s < L; ++s) {
    const int a = s % 3, lev = s / 3;
    double rot[2][2][2];   // [b][row][col]
    for (int b = 0; b < 2; ++b) {
      const double th = 2.0 * M_PI * row[a] * (double)(1 << (n_bits - 1 - lev)) * b / N;
      rot[b][0][0] = cos(th); rot[b][0][1] = sin(th);
      rot[b][1][0] = -sin(th); rot[b][1][1] = cos(th);
    }
    const int r0 = s == 0 ? 1 : 2, r1 = s == L - 1 ? 1 : 2;
    std::vector<double>& c = cores[s];
    c.assign((size_t)r0 * 2 * r1, 0.0);
    for (int i = 0; i < r0; ++i)
      for (int b = 0; b < 2; ++b)
        for (int jj = 0; jj < r1; ++jj) {
          double v;
          if (s == 0) v = cos(row[3]) * rot[b][0][jj] + sin(row[3]) * rot[b][1][jj];
          else v = rot[b][i][jj];
          c[((size_t)i * 2 + b) * r1 + jj] = v;
        }
  }
}

template <typename T>
static int upload_host_mps(tnlbm_sim* s, int node, const double* cores, const int* ranks, int cap_src) {
  const MpsRef& m = s->nodes[node];
  std::vector<T> buf(mps_size(s->L, m.cap), (T)0);
  for (int k = 0; k < s->L; ++k) {
    const int r0 = ranks[k], r1 = ranks[k + 1];
    if (r0 > bond_cap(s->L, m.cap, k) || r1 > bond_cap(s->L, m.cap, k + 1) || r0 < 1 || r1 < 1) {
      set_error("MPS bond exceeds capacity");
      return TNLBM_E_CAPACITY;
    }
    const double* src = cores + core_offset(s->L, cap_src, k);
    T* dst = buf.data() + core_offset(s->L, m.cap, k);
    for (int i = 0; i < r0 * 2 * r1; ++i) dst[i] = (T)src[i];
  }
  TN_CUDA(cudaMemcpy(m.base, buf.data(), buf.size() * sizeof(T), cudaMemcpyHostToDevice));
  TN_CUDA(cudaMemcpy(m.ranks, ranks, (s->L + 1) * sizeof(int), cudaMemcpyHostToDevice));
  return 0;
}

template <typename T>
static int create_impl(tnlbm_sim* s) {
  tnlbm_config& C = s->cfg;
  TN_CUDA(cudaStreamCreateWithFlags(&s->s0, cudaStreamNonBlocking));
  TN_CUDA(cudaStreamCreateWithFlags(&s->s1, cudaStreamNonBlocking));
  TN_CUDA(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
  TN_CUDA(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
  s->d_scal = (double*)s->arena.alloc(SC_COUNT * sizeof(double));
  s->d_status = (int*)s->arena.alloc(STATUS_INTS * sizeof(int));
  s->d_discard = (double*)s->arena.alloc(sizeof(double));
  if (!s->d_scal || !s->d_status || !s->d_discard) return TNLBM_E_OOM;
  cudaMemset(s->d_scal, 0, SC_COUNT * sizeof(double));
  cudaMemset(s->d_discard, 0, sizeof(double));
  {
    double ub[18] = {0};                     // inlet velocities of the velocity faces
    for (int f6 = 0; f6 < 6; ++f6)
      if (C.face_kind[f6] == TNLBM_FACE_VELOCITY)
        for (int d = 0; d < 3; ++d) ub[3 * f6 + d] = C.face_u[f6][d];
    cudaMemcpy(s->d_scal + SC_UBRAW, ub, sizeof(ub), cudaMemcpyHostToDevice);
  }
  cudaMemset(s->d_status, 0, STATUS_INTS * sizeof(int));
  const int Q = s->lat.Q;
  // state
  for (int i = 0; i < Q; ++i) {
    int id = new_node(s, C.chi_max, 0);
    if (id < 0) return TNLBM_E_OOM;
    s->f_state.push_back(id);
  }
  // mask m_O
  const size_t ncell = (size_t)s->N * s->N * s->N;
  if (C.mask_cores || C.solid) {
    const int mcap = C.mask_cores ? C.mask_cap : std::max(1, C.chi_mask);
    s->mask_node = new_node(s, mcap, 0);
    if (s->mask_node < 0) return TNLBM_E_OOM;
    if (C.mask_cores) {
      int rc = upload_host_mps<T>(s, s->mask_node, C.mask_cores, C.mask_ranks, C.mask_cap);
      if (rc) return rc;
    } else {
      std::vector<T> h(ncell);
      for (size_t i = 0; i < ncell; ++i) h[i] = (T)(C.solid[i] ? 1 : 0);
      T* d = nullptr;
      TN_CUDA(cudaMalloc(&d, ncell * sizeof(T)));
      cudaMemcpy(d, h.data(), ncell * sizeof(T), cudaMemcpyHostToDevice);
      const MpsRef& m = s->nodes[s->mask_node];
      int rc = tt_svd_dense<T>(d, s->n, (T*)m.base, m.ranks, m.cap, m.cap, C.eps_mask, s->d_status, s->s0);
      cudaFree(d);
      if (rc) return rc;
    }
    // N_fluid = N^3 - <m_O, 1>
    MpsRef* dref = (MpsRef*)s->arena.alloc(sizeof(MpsRef));
    double* dout = (double*)s->arena.alloc(sizeof(double));
    cudaMemcpy(dref, &s->nodes[s->mask_node], sizeof(MpsRef), cudaMemcpyHostToDevice);
    launch_inner_ones<T>(dref, 1, s->L, dout, s->s0);
    double hm = 0.0;
    cudaMemcpyAsync(&hm, dout, sizeof(double), cudaMemcpyDeviceToHost, s->s0);
    TN_CUDA(cudaStreamSynchronize(s->s0));
    s->n_fluid = (double)ncell - hm;
  } else {
    s->n_fluid = (double)ncell;
  }
  // initial populations
  {
    std::vector<RoundJob> jobs(Q);
    std::vector<int> mode_nodes;
    if (C.n_modes > 0) {
      if (C.n_modes + 1 > TN_MAXT) { set_error("n_modes too large"); return TNLBM_E_ARG; }
      std::vector<std::vector<double>> cores;
      for (int m = 0; m < C.n_modes; ++m) {
        int id = new_node(s, 2, 0);
        if (id < 0) return TNLBM_E_OOM;
        mode_cores(s->n, C.modes + 8 * m, cores);
        std::vector<double> flat(mps_size(s->L, 2), 0.0);
        std::vector<int> rk(s->L + 1, 2);
        rk[0] = 1; rk[s->L] = 1;
        for (int k = 0; k < s->L; ++k)
          std::copy(cores[k].begin(), cores[k].end(), flat.begin() + core_offset(s->L, 2, k));
        int rc = upload_host_mps<T>(s, id, flat.data(), rk.data(), 2);
        if (rc) return rc;
        mode_nodes.push_back(id);
      }
    }
    for (int i = 0; i < Q; ++i) {
      RoundJob& j = jobs[i];
      j = RoundJob{};
      j.chi = C.chi_max; j.eps = C.eps;
      j.dst = s->nodes[s->f_state[i]];
      const double w = s->lat.w[i];
      int t = 0;
      j.t[t] = Term{}; j.t[t].kind = T_ONES; j.t[t].coef = w; j.t[t].coef_slot = -1; ++t;
      if (C.n_modes > 0) {
        for (int m = 0; m < C.n_modes; ++m) {
          const double* row = C.modes + 8 * m;
          double cu = 0.0;
          for (int d = 0; d < 3; ++d) cu += s->lat.c[i][d] * row[5 + d];
          j.t[t] = Term{}; j.t[t].kind = T_PLAIN; j.t[t].x = s->nodes[mode_nodes[m]];
          j.t[t].coef = w * (row[4] + 3.0 * cu); j.t[t].coef_slot = -1; ++t;
        }
      } else if (s->mask_node >= 0) {
        j.t[t] = Term{}; j.t[t].kind = T_PLAIN; j.t[t].x = s->nodes[s->mask_node];
        j.t[t].coef = -w; j.t[t].coef_slot = -1; ++t;
      }
      j.nterms = t;
    }
    int rc = run_round_now<T>(s, jobs);
    if (rc) return rc;
  }
  // the step DAG
  Builder b{s};
  b.build_step();
  if (b.oom) { set_error("out of device memory building the step"); return TNLBM_E_OOM; }
  s->d_masks = s->arena.alloc(std::max<size_t>(s->mask_vecs.size(), 2) * sizeof(T));
  {
    std::vector<T> mv(std::max<size_t>(s->mask_vecs.size(), 2), (T)0);
    for (size_t i = 0; i < s->mask_vecs.size(); ++i) mv[i] = (T)s->mask_vecs[i];
    cudaMemcpy(s->d_masks, mv.data(), mv.size() * sizeof(T), cudaMemcpyHostToDevice);
  }
  s->d_rho_ref = (MpsRef*)s->arena.alloc(sizeof(MpsRef));
  cudaMemcpy(s->d_rho_ref, &s->nodes[s->rho_node], sizeof(MpsRef), cudaMemcpyHostToDevice);
  {
    std::vector<MpsRef> src, dst;
    for (int i = 0; i < Q; ++i) { src.push_back(s->nodes[s->f_next[i]]); dst.push_back(s->nodes[s->f_state[i]]); }
    s->d_copy_src = (MpsRef*)s->arena.alloc(Q * sizeof(MpsRef));
    s->d_copy_dst = (MpsRef*)s->arena.alloc(Q * sizeof(MpsRef));
    cudaMemcpy(s->d_copy_src, src.data(), Q * sizeof(MpsRef), cudaMemcpyHostToDevice);
    cudaMemcpy(s->d_copy_dst, dst.data(), Q * sizeof(MpsRef), cudaMemcpyHostToDevice);
  }
  int rc = upload_levels<T>(s);
  if (rc) return rc;
  // initial mass, for the optional mass correction
  s->d_mass = (double*)s->arena.alloc(Q * sizeof(double));
  s->d_mass0 = (double*)s->arena.alloc(sizeof(double));
  if (!s->d_mass || !s->d_mass0) return TNLBM_E_OOM;
  {
    MpsRef* dref = (MpsRef*)s->arena.alloc(Q * sizeof(MpsRef));
    std::vector<MpsRef> refs;
    for (int i = 0; i < Q; ++i) refs.push_back(s->nodes[s->f_state[i]]);
    cudaMemcpy(dref, refs.data(), Q * sizeof(MpsRef), cudaMemcpyHostToDevice);
    launch_inner_ones<T>(dref, Q, s->L, s->d_mass, s->s0);
    std::vector<double> hm(Q);
    cudaMemcpyAsync(hm.data(), s->d_mass, Q * sizeof(double), cudaMemcpyDeviceToHost, s->s0);
    TN_CUDA(cudaStreamSynchronize(s->s0));
    double m0 = 0.0;
    for (double v : hm) m0 += v;
    cudaMemcpy(s->d_mass0, &m0, sizeof(double), cudaMemcpyHostToDevice);
  }
  rc = capture_graph<T>(s);
  if (rc) return rc;
  int st[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpy(st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[0]) return status_to_code(st);
  return 0;
}

}  // namespace tn

// ================================================================ C ABI
extern "C" {

const char* tnlbm_last_error(void) { return tn::g_err.c_str(); }

size_t tnlbm_mps_size(int L, int cap) { return tn::mps_size(L, cap); }
size_t tnlbm_mps_offset(int L, int cap, int k) { return tn::core_offset(L, cap, k); }

int tnlbm_create(const tnlbm_config* cfg, tnlbm_sim** out) {
  if (!out) { set_error("out is NULL"); return TNLBM_E_ARG; }
  *out = nullptr;
  if (!cfg) { set_error("cfg is NULL"); return TNLBM_E_ARG; }
  const tnlbm_config& C = *cfg;
  if (C.n_per_axis < 1 || C.n_per_axis > 10) { set_error("n_per_axis must be in [1, 10]"); return TNLBM_E_ARG; }
  if (C.lattice != TNLBM_D3Q19 && C.lattice != TNLBM_D3Q15) { set_error("lattice must be 19 or 15"); return TNLBM_E_ARG; }
  if (!(C.tau > 0.5)) { set_error("tau must exceed 0.5"); return TNLBM_E_ARG; }
  if (C.chi_max < 1 || C.chi_max > 512) { set_error("chi_max must be in [1, 512]"); return TNLBM_E_ARG; }
  if (C.eps < 0.0) { set_error("eps must be >= 0"); return TNLBM_E_ARG; }
  if (C.precision != TNLBM_FP64 && C.precision != TNLBM_FP32 && C.precision != TNLBM_TF32 &&
      C.precision != TNLBM_MIXED && C.precision != TNLBM_BF16) {
    set_error("bad precision");
    return TNLBM_E_ARG;
  }
  if (C.jacobi_max_sweeps < 0 || C.wait_limit_ns < 0 || C.max_cluster < 0 || C.max_cluster > 16) {
    set_error("jacobi_max_sweeps, wait_limit_ns >= 0; max_cluster in 0..16");
    return TNLBM_E_ARG;
  }
  if (C.learned_rank != 0 && C.learned_rank != 1 && C.learned_rank != 3) {
    set_error("learned_rank must be 0, 1 or 3 (the rank model is set with tnlbm_learn_set_mlp)");
    return TNLBM_E_ARG;
  }
  if (C.hadamard != TNLBM_HADAMARD_FIT && C.hadamard != TNLBM_HADAMARD_EXACT && C.hadamard != TNLBM_HADAMARD_ZIPUP) {
    set_error("bad hadamard mode");
    return TNLBM_E_ARG;
  }
  if (C.hadamard == TNLBM_HADAMARD_ZIPUP && C.chi_max > 512) { set_error("zip-up products need chi_max <= 512"); return TNLBM_E_ARG; }
  if (C.solid && C.mask_cores) { set_error("give solid voxels or mask cores, not both"); return TNLBM_E_ARG; }
  if (C.mask_cores && (!C.mask_ranks || C.mask_cap < 1)) { set_error("mask_ranks / mask_cap missing"); return TNLBM_E_ARG; }
  if (C.solid && (C.chi_mask < 1 || C.chi_mask > 512)) { set_error("chi_mask must be in [1, 512]"); return TNLBM_E_ARG; }
  if (C.n_modes < 0 || (C.n_modes > 0 && !C.modes)) { set_error("modes missing"); return TNLBM_E_ARG; }
  if (C.block_sums && (C.lattice * C.chi_max > 1024)) {
    set_error("block_sums needs Q * chi_max <= 1024 (the summed bond of one rounding)");
    return TNLBM_E_ARG;
  }
  for (int f6 = 0; f6 < 6; ++f6) {
    const int k = C.face_kind[f6];
    if (k < TNLBM_FACE_WALL || k > TNLBM_FACE_PRESSURE) { set_error("bad face_kind"); return TNLBM_E_ARG; }
    if (k != TNLBM_FACE_WALL && C.periodic[f6 / 2]) {
      set_error("inlet / outlet faces need a non-periodic axis");
      return TNLBM_E_ARG;
    }
    if (k == TNLBM_FACE_PRESSURE && !(C.face_rho[f6] > 0.0)) { set_error("face_rho must be > 0"); return TNLBM_E_ARG; }
  }
  tnlbm_sim* s = new (std::nothrow) tnlbm_sim();
  if (!s) { set_error("host allocation failed"); return TNLBM_E_OOM; }
  s->n = C.n_per_axis;
  s->L = 3 * s->n;
  s->N = 1 << s->n;
  s->prec = C.precision;
  s->esz = C.precision == TNLBM_FP64 ? 8 : 4;
  s->lat = make_lattice(C.lattice);
  s->cfg = C;              // pointers are used during create only
  if (s->cfg.sweeps <= 0) s->cfg.sweeps = 2;
  int rc = C.precision == TNLBM_FP64 ? tn::create_impl<double>(s) : tn::create_impl<float>(s);
  s->cfg.solid = nullptr;
  s->cfg.mask_cores = nullptr;
  s->cfg.mask_ranks = nullptr;
  s->cfg.modes = nullptr;
  if (!rc && C.learned_rank > 0) {
    // Gaussian test matrix of the randomized truncation from the seed:
    // SplitMix64 uniforms in (0, 1], Box-Muller pairs
    const int rows = 2 * C.chi_max, ld = C.chi_max + 8;
    std::vector<double> om((size_t)rows * ld);
    uint64_t x = C.seed;
    auto next = [&x]() {
      uint64_t z = (x += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return ((double)(z >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    };
    for (size_t i = 0; i < om.size(); i += 2) {
      const double u1 = next(), u2 = next();
      const double rad = std::sqrt(-2.0 * std::log(u1)), th = 6.283185307179586 * u2;
      om[i] = rad * std::cos(th);
      if (i + 1 < om.size()) om[i + 1] = rad * std::sin(th);
    }
    rc = tnlbm_learn_configure(s, C.learned_rank, om.data(), rows, ld, 8, 1, 0.2,
                               C.precision == TNLBM_FP64 ? 1e-12 : 1e-5, C.learned_rank == 1 ? 65536 : 0);
  }
  if (rc) {
    std::string msg = tn::g_err;
    tnlbm_destroy(s);
    tn::g_err = msg;
    return rc;
  }
  *out = s;
  return 0;
}

int tnlbm_step(tnlbm_sim* s, int k) {
  if (!s || k < 0) { set_error("bad arguments to tnlbm_step"); return TNLBM_E_ARG; }
  for (int i = 0; i < k; ++i) TN_CUDA(cudaGraphLaunch(s->gexec, s->s0));
  TN_CUDA(cudaStreamSynchronize(s->s0));
  s->steps += k;
  int st[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpy(st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[0]) {
    int rc = status_to_code(st);
    cudaMemset(s->d_status, 0, STATUS_INTS * sizeof(int));
    return rc;
  }
  return 0;
}

}  // extern "C"

namespace tn {

template <typename LV>
static int get_clusters(const std::vector<LV>& levels, int* clusters, int* jobs, int cap, int* nlevels) {
  const int n = (int)levels.size();
  for (int l = 0; l < std::min(std::max(cap, 0), n); ++l) {
    if (clusters) clusters[l] = levels[l].rj.empty() ? 0 : levels[l].cluster;
    if (jobs) jobs[l] = (int)levels[l].rj.size();
  }
  if (nlevels) *nlevels = n;
  return 0;
}

template <typename T, typename LV>
static int set_clusters(std::vector<LV>& levels, int prec, const int* clusters, int nlevels) {
  if (!clusters || nlevels != (int)levels.size()) {
    set_error("setting cluster sizes needs one entry per dependency level (" + std::to_string(levels.size()) + ")");
    return TNLBM_E_ARG;
  }
  for (int l = 0; l < nlevels; ++l)
    if (!levels[l].rj.empty()) {
      const int rc = check_cluster<T>(prec, clusters[l]);
      if (rc) return rc;
    }
  for (int l = 0; l < nlevels; ++l)
    if (!levels[l].rj.empty()) levels[l].cluster = clusters[l];
  return 0;
}

}  // namespace tn

extern "C" {

int tnlbm_clusters(tnlbm_sim* s, int* clusters, int* jobs, int cap, int* nlevels) {
  if (!s) { set_error("bad arguments to tnlbm_clusters"); return TNLBM_E_ARG; }
  return tn::get_clusters(s->levels, clusters, jobs, cap, nlevels);
}

int tnlbm_set_clusters(tnlbm_sim* s, const int* clusters, int nlevels) {
  if (!s) { set_error("bad arguments to tnlbm_set_clusters"); return TNLBM_E_ARG; }
  const bool f64 = s->prec == TNLBM_FP64;
  int rc = f64 ? tn::set_clusters<double>(s->levels, s->prec, clusters, nlevels)
               : tn::set_clusters<float>(s->levels, s->prec, clusters, nlevels);
  if (rc) return rc;
  return f64 ? tn::capture_graph<double>(s) : tn::capture_graph<float>(s);
}

int tnlbm_tune_clusters(tnlbm_sim* s, int reps, double* ms, int ms_cap) {
  if (!s || reps < 1 || (ms && ms_cap < 0)) { set_error("bad arguments to tnlbm_tune_clusters"); return TNLBM_E_ARG; }
  return s->prec == TNLBM_FP64 ? tn::tune_sim<double>(s, reps, ms, ms_cap) : tn::tune_sim<float>(s, reps, ms, ms_cap);
}

}  // extern "C"

template <typename T>
static int macro_impl(tnlbm_sim* s, double* rho, double* u) {
  using namespace tn;
  const size_t nc = (size_t)s->N * s->N * s->N;
  double *d = nullptr, *dm = nullptr, *tmp = nullptr;
  void* scr = nullptr;
  const int capmax = std::max(s->cfg.chi_max, s->mask_node >= 0 ? s->nodes[s->mask_node].cap : 1);
  const size_t sb = contract_scratch_bytes(s->n, capmax, sizeof(T));
  auto fin = [&](int rc) { cudaFree(d); cudaFree(dm); cudaFree(tmp); cudaFree(scr); return rc; };
  if (cudaMalloc(&d, 4 * nc * sizeof(double)) != cudaSuccess || cudaMalloc(&tmp, nc * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&scr, sb) != cudaSuccess) {
    set_error("out of device memory in tnlbm_macroscopic");
    return fin(TNLBM_E_OOM);
  }
  double *dr = d, *jx = d + nc, *jy = d + 2 * nc, *jz = d + 3 * nc;
  for (int i = 0; i < s->lat.Q; ++i) {
    contract_dense_f64<T>(s->nodes[s->f_state[i]], s->n, tmp, scr, sb, s->s0);
    launch_accum_moments<double>(tmp, nc, dr, jx, jy, jz, s->lat.c[i][0], s->lat.c[i][1], s->lat.c[i][2], i == 0, s->s0);
  }
  if (s->mask_node >= 0) {
    if (cudaMalloc(&dm, nc * sizeof(double)) != cudaSuccess) return fin(TNLBM_E_OOM);
    contract_dense_f64<T>(s->nodes[s->mask_node], s->n, dm, scr, sb, s->s0);
  }
  if (u) launch_velocity(nc, dr, jx, jy, jz, dm, s->cfg.force[0], s->cfg.force[1], s->cfg.force[2], s->s0);
  if (rho) cudaMemcpyAsync(rho, dr, nc * sizeof(double), cudaMemcpyDeviceToHost, s->s0);
  if (u) cudaMemcpyAsync(u, jx, 3 * nc * sizeof(double), cudaMemcpyDeviceToHost, s->s0);
  cudaError_t e = cudaStreamSynchronize(s->s0);
  if (e != cudaSuccess) return fin(cuda_fail(e, "tnlbm_macroscopic"));
  return fin(0);
}

template <typename T>
static int slice_impl(tnlbm_sim* s, int axis, int index, double* rho, double* u) {
  using namespace tn;
  const size_t nc = (size_t)s->N * s->N;
  double *d = nullptr, *dm = nullptr, *tmp = nullptr;
  void* scr = nullptr;
  const int capmax = std::max(s->cfg.chi_max, s->mask_node >= 0 ? s->nodes[s->mask_node].cap : 1);
  const size_t sb = plane_scratch_bytes(s->n, axis, capmax);
  auto fin = [&](int rc) { cudaFree(d); cudaFree(dm); cudaFree(tmp); cudaFree(scr); return rc; };
  if (cudaMalloc(&d, 4 * nc * sizeof(double)) != cudaSuccess || cudaMalloc(&tmp, nc * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&scr, sb) != cudaSuccess) {
    set_error("out of device memory in tnlbm_macroscopic_slice");
    return fin(TNLBM_E_OOM);
  }
  double *dr = d, *jx = d + nc, *jy = d + 2 * nc, *jz = d + 3 * nc;
  for (int i = 0; i < s->lat.Q; ++i) {
    contract_plane_f64<T>(s->nodes[s->f_state[i]], s->n, axis, index, tmp, scr, sb, s->s0);
    launch_accum_moments<double>(tmp, nc, dr, jx, jy, jz, s->lat.c[i][0], s->lat.c[i][1], s->lat.c[i][2], i == 0, s->s0);
  }
  if (s->mask_node >= 0) {
    if (cudaMalloc(&dm, nc * sizeof(double)) != cudaSuccess) return fin(TNLBM_E_OOM);
    contract_plane_f64<T>(s->nodes[s->mask_node], s->n, axis, index, dm, scr, sb, s->s0);
  }
  if (u) launch_velocity(nc, dr, jx, jy, jz, dm, s->cfg.force[0], s->cfg.force[1], s->cfg.force[2], s->s0);
  if (rho) cudaMemcpyAsync(rho, dr, nc * sizeof(double), cudaMemcpyDeviceToHost, s->s0);
  if (u) cudaMemcpyAsync(u, jx, 3 * nc * sizeof(double), cudaMemcpyDeviceToHost, s->s0);
  cudaError_t e = cudaStreamSynchronize(s->s0);
  if (e != cudaSuccess) return fin(cuda_fail(e, "tnlbm_macroscopic_slice"));
  return fin(0);
}

template <typename T>
static int get_pop_impl(tnlbm_sim* s, double* cores, int* ranks) {
  using namespace tn;
  const size_t ms = mps_size(s->L, s->cfg.chi_max);
  std::vector<T> buf(ms);
  for (int i = 0; i < s->lat.Q; ++i) {
    const MpsRef& m = s->nodes[s->f_state[i]];
    TN_CUDA(cudaMemcpy(buf.data(), m.base, ms * sizeof(T), cudaMemcpyDeviceToHost));
    if (cores) for (size_t e = 0; e < ms; ++e) cores[(size_t)i * ms + e] = (double)buf[e];
    if (ranks) TN_CUDA(cudaMemcpy(ranks + (size_t)i * (s->L + 1), m.ranks, (s->L + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  }
  return 0;
}

template <typename T>
static int set_pop_impl(tnlbm_sim* s, const double* cores, const int* ranks) {
  using namespace tn;
  const size_t ms = mps_size(s->L, s->cfg.chi_max);
  for (int i = 0; i < s->lat.Q; ++i) {
    int rc = upload_host_mps<T>(s, s->f_state[i], cores + (size_t)i * ms, ranks + (size_t)i * (s->L + 1), s->cfg.chi_max);
    if (rc) return rc;
  }
  return 0;
}

extern "C" {

int tnlbm_macroscopic(tnlbm_sim* s, double* rho, double* u) {
  if (!s) { set_error("sim is NULL"); return TNLBM_E_ARG; }
  return s->prec == TNLBM_FP64 ? macro_impl<double>(s, rho, u) : macro_impl<float>(s, rho, u);
}

int tnlbm_macroscopic_slice(tnlbm_sim* s, int axis, int index, double* rho, double* u) {
  if (!s || axis < 0 || axis > 2 || index < 0 || index >= s->N) {
    set_error("bad arguments to tnlbm_macroscopic_slice");
    return TNLBM_E_ARG;
  }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  return s->prec == TNLBM_FP64 ? slice_impl<double>(s, axis, index, rho, u) : slice_impl<float>(s, axis, index, rho, u);
}

int tnlbm_get_populations(tnlbm_sim* s, double* cores, int* ranks) {
  if (!s) { set_error("sim is NULL"); return TNLBM_E_ARG; }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  return s->prec == TNLBM_FP64 ? get_pop_impl<double>(s, cores, ranks) : get_pop_impl<float>(s, cores, ranks);
}

int tnlbm_set_populations(tnlbm_sim* s, const double* cores, const int* ranks) {
  if (!s || !cores || !ranks) { set_error("NULL argument"); return TNLBM_E_ARG; }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  return s->prec == TNLBM_FP64 ? set_pop_impl<double>(s, cores, ranks) : set_pop_impl<float>(s, cores, ranks);
}

int tnlbm_stats_get(tnlbm_sim* s, tnlbm_stats* out) {
  if (!s || !out) { set_error("NULL argument"); return TNLBM_E_ARG; }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  std::vector<int> rk((size_t)s->lat.Q * (s->L + 1));
  for (int i = 0; i < s->lat.Q; ++i)
    TN_CUDA(cudaMemcpy(rk.data() + (size_t)i * (s->L + 1), s->nodes[s->f_state[i]].ranks, (s->L + 1) * sizeof(int),
                       cudaMemcpyDeviceToHost));
  int mx = 0;
  double sum = 0.0, nv = 0.0;
  int cnt = 0;
  for (int i = 0; i < s->lat.Q; ++i)
    for (int k = 0; k <= s->L; ++k) {
      int r = rk[(size_t)i * (s->L + 1) + k];
      mx = std::max(mx, r);
      if (k > 0 && k < s->L) { sum += r; ++cnt; }
      if (k < s->L) nv += (double)r * 2.0 * rk[(size_t)i * (s->L + 1) + k + 1];
    }
  double scal[SC_COUNT] = {0};
  TN_CUDA(cudaMemcpy(scal, s->d_scal, sizeof(scal), cudaMemcpyDeviceToHost));
  int st = 0;
  TN_CUDA(cudaMemcpy(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  out->steps = s->steps;
  out->max_bond = mx;
  out->mean_bond = cnt ? sum / cnt : 0.0;
  out->nvps = nv;
  out->compression_ratio = nv > 0 ? (double)s->lat.Q * s->N * s->N * s->N / nv : 0.0;
  out->rho0 = scal[SC_RHO0];
  out->status = st;
  out->gpu_launches_per_step = s->launches_per_step;
  double disc = 0.0;
  TN_CUDA(cudaMemcpy(&disc, s->d_discard, sizeof(double), cudaMemcpyDeviceToHost));
  out->discarded2 = disc;
  out->mass = scal[SC_RHO0] * s->n_fluid;
  out->round_jobs_per_step = 0;
  out->product_jobs_per_step = 0;
  out->round_ctas_per_step = 0;
  out->max_cluster = 1;
  for (auto& lv : s->levels) {
    out->round_jobs_per_step += (int)lv.rj.size();
    out->product_jobs_per_step += (int)(lv.fj.size() + lv.zj.size());
    out->round_ctas_per_step += (int)lv.rj.size() * lv.cluster;
    out->max_cluster = std::max(out->max_cluster, lv.cluster);
  }
  return 0;
}

int tnlbm_learn_configure(tnlbm_sim* s, int mode, const double* omega, int omega_rows, int omega_ld,
                          int oversample, int power, double eta, double floor_rel, int dataset_cap) {
  if (!s || mode < 0 || mode > 3 ||
      (mode > 0 && (!omega || omega_rows < 2 * s->cfg.chi_max || omega_ld < 1 || oversample < 0 ||
                    power < 0 || power > 4 || !(eta > 0.0) || !(eta < 1.0) || floor_rel < 0.0 ||
                    dataset_cap < 0))) {
    set_error("bad arguments to tnlbm_learn_configure");
    return TNLBM_E_ARG;
  }
  if (mode == 2 && !s->mlp_set) {
    set_error("tnlbm_learn_configure: mode 2 needs a rank model (tnlbm_learn_set_mlp)");
    return TNLBM_E_ARG;
  }
  return s->prec == TNLBM_FP64
             ? tn::learn_configure_impl<double>(s, mode, omega, omega_rows, omega_ld, oversample, power, eta, floor_rel, dataset_cap)
             : tn::learn_configure_impl<float>(s, mode, omega, omega_rows, omega_ld, oversample, power, eta, floor_rel, dataset_cap);
}

int tnlbm_learn_set_mlp(tnlbm_sim* s, const void* params_f16) {
  if (!s || !params_f16) { set_error("bad arguments to tnlbm_learn_set_mlp"); return TNLBM_E_ARG; }
  if (!s->d_learn) {
    // allocate the learning state (mode stays off)
    std::vector<double> om(2 * (size_t)s->cfg.chi_max, 0.0);
    int rc = s->prec == TNLBM_FP64
                 ? tn::learn_configure_impl<double>(s, 0, om.data(), 2 * s->cfg.chi_max, 1, 0, 0, 0.5, 0.0, 0)
                 : tn::learn_configure_impl<float>(s, 0, om.data(), 2 * s->cfg.chi_max, 1, 0, 0, 0.5, 0.0, 0);
    if (rc) return rc;
  }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  TN_CUDA(cudaMemcpy(s->d_mlp, params_f16, tn::MLP_NPARAM * sizeof(__half), cudaMemcpyDefault));
  s->mlp_set = true;
  return 0;
}

int tnlbm_learn_dataset(tnlbm_sim* s, float* out, int cap, int* count, int reset) {
  if (!s || cap < 0 || (cap > 0 && !out) || !count) { set_error("bad arguments to tnlbm_learn_dataset"); return TNLBM_E_ARG; }
  *count = 0;
  if (!s->d_learn) return 0;
  TN_CUDA(cudaStreamSynchronize(s->s0));
  int hc[4] = {0};
  TN_CUDA(cudaMemcpy(hc, s->d_lcount, sizeof(hc), cudaMemcpyDeviceToHost));
  const int stored = std::min(hc[3], s->h_learn.dataset_cap);
  const int n = std::min(stored, cap);
  if (n > 0)
    TN_CUDA(cudaMemcpy(out, s->d_dataset, (size_t)n * (tn::MLP_IN + 1) * sizeof(float), cudaMemcpyDefault));
  *count = hc[3];
  if (reset) TN_CUDA(cudaMemset(s->d_lcount + 3, 0, sizeof(int)));
  return 0;
}

int tnlbm_learn_counters(tnlbm_sim* s, long long* out, int reset) {
  if (!s || !out) { set_error("bad arguments to tnlbm_learn_counters"); return TNLBM_E_ARG; }
  out[0] = out[1] = out[2] = 0;
  if (!s->d_learn) return 0;
  TN_CUDA(cudaStreamSynchronize(s->s0));
  int hc[4] = {0};
  TN_CUDA(cudaMemcpy(hc, s->d_lcount, sizeof(hc), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 3; ++i) out[i] = hc[i];
  if (reset) TN_CUDA(cudaMemset(s->d_lcount, 0, 3 * sizeof(int)));
  return 0;
}

int tnlbm_set_limits(tnlbm_sim* s, int jacobi_max_sweeps, long long wait_limit_ns) {
  if (!s || jacobi_max_sweeps < 0 || wait_limit_ns < 0) {
    set_error("bad arguments to tnlbm_set_limits");
    return TNLBM_E_ARG;
  }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  s->cfg.jacobi_max_sweeps = jacobi_max_sweeps;
  s->cfg.wait_limit_ns = wait_limit_ns;
  for (auto& lv : s->levels) {
    if (lv.rj.empty()) continue;
    for (auto& rj : lv.rj) {
      rj.max_sweeps = jacobi_max_sweeps;
      rj.wait_ns = wait_limit_ns;
    }
    TN_CUDA(cudaMemcpy(lv.d_rj, lv.rj.data(), lv.rj.size() * sizeof(RoundJob), cudaMemcpyHostToDevice));
  }
  return 0;
}

int tnlbm_set_face_velocity(tnlbm_sim* s, int face, const double* u) {
  if (!s || face < 0 || face > 5 || !u) { set_error("bad arguments to tnlbm_set_face_velocity"); return TNLBM_E_ARG; }
  if (s->cfg.face_kind[face] != TNLBM_FACE_VELOCITY) {
    set_error("tnlbm_set_face_velocity: the face is not a velocity face");
    return TNLBM_E_ARG;
  }
  TN_CUDA(cudaStreamSynchronize(s->s0));
  TN_CUDA(cudaMemcpy(s->d_scal + SC_UBRAW + 3 * face, u, 3 * sizeof(double), cudaMemcpyHostToDevice));
  for (int d = 0; d < 3; ++d) s->cfg.face_u[face][d] = u[d];
  return 0;
}

int tnlbm_destroy(tnlbm_sim* s) {
  if (!s) return 0;
  if (s->s0) cudaStreamSynchronize(s->s0);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->s0) cudaStreamDestroy(s->s0);
  if (s->s1) cudaStreamDestroy(s->s1);
  delete s;
  return 0;
}

}  // extern "C"

// ================================================================ primitives
namespace tn {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  bool alloc(size_t b) { return cudaMalloc(&p, b ? b : 16) == cudaSuccess; }
};

static int check_status(int* d_status, cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "primitive");
  int h[STATUS_INTS] = {0};
  e = cudaMemcpy(h, d_status, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  return status_to_code(h);
}

struct RsvdArgs {               // randomized truncation at given target ranks
  const int* targets;           // host, batch x (L + 1); 0 = full SVD at that bond
  const void* omega;            // device, element type of the rounding, rows x ld
  int rows, ld, oversample, power;
  double eta, floor_rel;
  int* counters;                // host [3]: accepted, fell back, full SVDs
};

template <typename T>
static int lincomb_impl(int n_bits, int batch, int nterms, const tnlbm_term* terms, void* const* dst,
                        int* const* dst_ranks, int dst_cap, int chi, double eps, int materialize,
                        cudaStream_t st, const RsvdArgs* ra = nullptr, int svd64 = 0) {
  const int L = 3 * n_bits;
  std::vector<RoundJob> jobs(batch);
  std::vector<T> masks;
  for (int b = 0; b < batch; ++b) {
    RoundJob& j = jobs[b];
    j = RoundJob{};
    j.svd64 = svd64;
    j.nterms = nterms;
    j.chi = chi;
    j.eps = eps;
    j.materialize_only = materialize;
    j.dst.base = dst[b];
    j.dst.ranks = dst_ranks[b];
    j.dst.cap = dst_cap;
    for (int t = 0; t < nterms; ++t) {
      const tnlbm_term& in = terms[(size_t)b * nterms + t];
      Term& tm = j.t[t];
      tm = Term{};
      tm.kind = in.kind;
      tm.coef = in.coef;
      tm.coef_slot = -1;
      tm.axis = in.axis;
      tm.offset = in.offset;
      tm.cyclic = in.cyclic;
      tm.mask_id = -1;
      if (in.kind < 0 || in.kind > 4) { set_error("bad term kind"); return TNLBM_E_ARG; }
      if (in.kind != T_ONES) {
        if (!in.x || !in.x_ranks || in.x_cap < 1) { set_error("term operand missing"); return TNLBM_E_ARG; }
        tm.x.base = (void*)in.x; tm.x.ranks = (int*)in.x_ranks; tm.x.cap = in.x_cap;
      }
      if (in.kind == T_KRON) {
        if (!in.y || !in.y_ranks || in.y_cap < 1) { set_error("KRON needs y"); return TNLBM_E_ARG; }
        tm.y.base = (void*)in.y; tm.y.ranks = (int*)in.y_ranks; tm.y.cap = in.y_cap;
      }
      if (in.kind == T_SHIFT && (in.axis < 0 || in.axis > 2 || (in.offset != 1 && in.offset != -1))) {
        set_error("SHIFT needs axis in 0..2 and offset +-1");
        return TNLBM_E_ARG;
      }
      if (in.kind == T_MASK1) {
        if (!in.mask) { set_error("MASK1 needs mask vectors"); return TNLBM_E_ARG; }
        tm.mask_id = (int)(masks.size() / (TN_MAXL * 2));
        masks.resize(masks.size() + TN_MAXL * 2, (T)1);
        for (int k = 0; k < L; ++k)
          for (int s2 = 0; s2 < 2; ++s2) masks[(size_t)tm.mask_id * TN_MAXL * 2 + 2 * k + s2] = (T)in.mask[2 * k + s2];
      }
    }
    plan_round_job(j, L, n_bits, sizeof(T));
  }
  size_t tot = 0;
  for (auto& j : jobs) tot += j.lay.total;
  DevBuf scr, dj, dm, ds, dsc, dtg, dlc, dcnt;
  if (!scr.alloc(tot * sizeof(T)) || !dj.alloc(batch * sizeof(RoundJob)) ||
      !dm.alloc(std::max<size_t>(masks.size(), 2) * sizeof(T)) || !ds.alloc(STATUS_INTS * sizeof(int)) ||
      !dsc.alloc(SC_COUNT * sizeof(double)) ||
      (ra && (!dtg.alloc((size_t)batch * (L + 1) * sizeof(int)) || !dlc.alloc(sizeof(LearnCtx)) ||
              !dcnt.alloc(4 * sizeof(int))))) {
    set_error("out of device memory");
    return TNLBM_E_OOM;
  }
  size_t o = 0;
  for (auto& j : jobs) { j.scratch = (T*)scr.p + o; o += j.lay.total; }
  if (ra) {
    for (int b = 0; b < batch; ++b) {
      jobs[b].rsvd_mode = 1;
      jobs[b].targets = (const int*)dtg.p + (size_t)b * (L + 1);
    }
    LearnCtx h{};
    h.omega = ra->omega;
    h.omega_rows = ra->rows;
    h.omega_ld = ra->ld;
    h.oversample = ra->oversample;
    h.power = ra->power;
    h.eta = (float)ra->eta;
    h.floor_rel = (float)ra->floor_rel;
    h.counters = (int*)dcnt.p;
    TN_CUDA(cudaMemcpyAsync(dtg.p, ra->targets, (size_t)batch * (L + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    TN_CUDA(cudaMemcpyAsync(dlc.p, &h, sizeof(LearnCtx), cudaMemcpyHostToDevice, st));
    TN_CUDA(cudaMemsetAsync(dcnt.p, 0, 4 * sizeof(int), st));
  }
  TN_CUDA(cudaMemcpyAsync(dj.p, jobs.data(), batch * sizeof(RoundJob), cudaMemcpyHostToDevice, st));
  if (!masks.empty()) TN_CUDA(cudaMemcpyAsync(dm.p, masks.data(), masks.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  TN_CUDA(cudaMemsetAsync(ds.p, 0, STATUS_INTS * sizeof(int), st));
  TN_CUDA(cudaMemsetAsync(dsc.p, 0, SC_COUNT * sizeof(double), st));
  const int cl = (!materialize && (svd64 || sizeof(T) == 8)) ? round_cluster_size<T>(batch, 16) : 1;
  launch_round<T>((const RoundJob*)dj.p, batch, L, n_bits, (const T*)dm.p, (const double*)dsc.p, (int*)ds.p, st,
                  nullptr, ra ? (const LearnCtx*)dlc.p : nullptr, cl);
  TN_CUDA(cudaGetLastError());
  int rc = check_status((int*)ds.p, st);
  if (ra && ra->counters) {
    int hc[4] = {0};
    TN_CUDA(cudaMemcpy(hc, dcnt.p, sizeof(hc), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 3; ++i) ra->counters[i] = hc[i];
  }
  return rc;
}

template <typename T>
static int fit_impl(int n_bits, int batch, int tc, const void* const* B, const int* const* rB, int capB,
                    const void* const* C, const int* const* rC, int capC, void* const* A,
                    int* const* rA, int capA, int sweeps, cudaStream_t st) {
  const int L = 3 * n_bits;
  std::vector<FitJob> jobs(batch);
  size_t tot = 0;
  for (int b = 0; b < batch; ++b) {
    FitJob& j = jobs[b];
    j = FitJob{};
    j.A.base = A[b]; j.A.ranks = rA[b]; j.A.cap = capA;
    j.B.base = (void*)B[b]; j.B.ranks = (int*)rB[b]; j.B.cap = capB;
    j.C.base = (void*)C[b]; j.C.ranks = (int*)rC[b]; j.C.cap = capC;
    size_t env, xs, ys, ab, q;
    plan_fit_job(j, L, &env, &xs, &ys, &ab, &q);
    j.env_stride = env;
    j.qscr_stride = q;
    tot += 2 * (L + 1) * env + xs + ys + ab + 4 * q;
  }
  DevBuf scr, dj, ds;
  if (!scr.alloc(tot * sizeof(T)) || !dj.alloc(batch * sizeof(FitJob)) || !ds.alloc(STATUS_INTS * sizeof(int))) {
    set_error("out of device memory");
    return TNLBM_E_OOM;
  }
  size_t o = 0;
  for (auto& j : jobs) {
    T* base = (T*)scr.p;
    size_t env, xs, ys, ab, q;
    plan_fit_job(j, L, &env, &xs, &ys, &ab, &q);
    j.env_l = base + o; o += (L + 1) * env;
    j.env_r = base + o; o += (L + 1) * env;
    j.x = base + o; o += xs;
    j.y = base + o; o += ys;
    j.abuf = base + o; o += ab;
    j.qscr = base + o; o += 4 * q;
  }
  TN_CUDA(cudaMemcpyAsync(dj.p, jobs.data(), batch * sizeof(FitJob), cudaMemcpyHostToDevice, st));
  TN_CUDA(cudaMemsetAsync(ds.p, 0, STATUS_INTS * sizeof(int), st));
  run_fit<T>((const FitJob*)dj.p, jobs, L, sweeps, (int*)ds.p, st, nullptr, tc);
  TN_CUDA(cudaGetLastError());
  return check_status((int*)ds.p, st);
}

template <typename T>
static int zipup_impl(int n_bits, int batch, const void* const* B, const int* const* rB, int capB,
                      const void* const* C, const int* const* rC, int capC, void* const* A, int* const* rA,
                      int capA, int chi, double eps, cudaStream_t st) {
  const int L = 3 * n_bits;
  std::vector<ZipJob> zj(batch);
  std::vector<RoundJob> rj(batch);
  const size_t zs = zip_scratch_elems(L, capB, capC, chi, sizeof(T));
  const size_t zm = mps_size(L, chi);
  DevBuf zscr, ztmp, zrk, dz, dr, ds, rscr;
  if (!zscr.alloc((size_t)batch * zs * sizeof(T)) || !ztmp.alloc((size_t)batch * zm * sizeof(T)) ||
      !zrk.alloc((size_t)batch * (L + 1) * sizeof(int)) || !dz.alloc(batch * sizeof(ZipJob)) ||
      !dr.alloc(batch * sizeof(RoundJob)) || !ds.alloc(STATUS_INTS * sizeof(int))) {
    set_error("out of device memory");
    return TNLBM_E_OOM;
  }
  size_t rtot = 0;
  for (int b = 0; b < batch; ++b) {
    ZipJob& z = zj[b];
    z = ZipJob{};
    z.B.base = (void*)B[b]; z.B.ranks = (int*)rB[b]; z.B.cap = capB;
    z.C.base = (void*)C[b]; z.C.ranks = (int*)rC[b]; z.C.cap = capC;
    z.Z.base = (T*)ztmp.p + (size_t)b * zm; z.Z.ranks = (int*)zrk.p + (size_t)b * (L + 1); z.Z.cap = chi;
    z.chi = chi;
    z.eps = eps;
    z.scratch = (T*)zscr.p + (size_t)b * zs;
    RoundJob& r = rj[b];
    r = RoundJob{};
    r.nterms = 1;
    r.chi = chi;
    r.eps = eps;
    r.t[0] = Term{};
    r.t[0].kind = T_PLAIN;
    r.t[0].coef = 1.0;
    r.t[0].coef_slot = -1;
    r.t[0].mask_id = -1;
    r.t[0].x = z.Z;
    r.dst.base = A[b]; r.dst.ranks = rA[b]; r.dst.cap = capA;
    plan_round_job(r, L, n_bits, sizeof(T));
    rtot += r.lay.total;
  }
  if (!rscr.alloc(rtot * sizeof(T))) { set_error("out of device memory"); return TNLBM_E_OOM; }
  size_t o = 0;
  for (auto& r : rj) { r.scratch = (T*)rscr.p + o; o += r.lay.total; }
  TN_CUDA(cudaMemcpyAsync(dz.p, zj.data(), batch * sizeof(ZipJob), cudaMemcpyHostToDevice, st));
  TN_CUDA(cudaMemcpyAsync(dr.p, rj.data(), batch * sizeof(RoundJob), cudaMemcpyHostToDevice, st));
  TN_CUDA(cudaMemsetAsync(ds.p, 0, STATUS_INTS * sizeof(int), st));
  run_zipup<T>((const ZipJob*)dz.p, batch, L, (int*)ds.p, st);
  launch_round<T>((const RoundJob*)dr.p, batch, L, n_bits, nullptr, nullptr, (int*)ds.p, st);
  TN_CUDA(cudaGetLastError());
  return check_status((int*)ds.p, st);
}

}  // namespace tn

extern "C" {

int tnlbm_lincomb_round(int precision, int n_bits, int batch, int nterms, const tnlbm_term* terms,
                        void* const* dst, int* const* dst_ranks, int dst_cap, int chi_max, double eps,
                        void* stream) {
  if (n_bits < 1 || n_bits > 10 || batch < 0 || nterms < 1 || nterms > TN_MAXT || !terms || !dst ||
      !dst_ranks || chi_max < 1 || chi_max > dst_cap || chi_max > 512 || eps < 0 || precision < TNLBM_FP64 ||
      precision > TNLBM_BF16) {
    set_error("bad arguments to tnlbm_lincomb_round");
    return TNLBM_E_ARG;
  }
  if (batch == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == TNLBM_FP64
             ? tn::lincomb_impl<double>(n_bits, batch, nterms, terms, dst, dst_ranks, dst_cap, chi_max, eps, 0, st)
             : tn::lincomb_impl<float>(n_bits, batch, nterms, terms, dst, dst_ranks, dst_cap, chi_max, eps, 0, st,
                                       nullptr, prec_svd64(precision) ? 1 : 0);
}

int tnlbm_lincomb_round_rsvd(int precision, int n_bits, int batch, int nterms, const tnlbm_term* terms,
                             void* const* dst, int* const* dst_ranks, int dst_cap, int chi_max, double eps,
                             const int* targets, const void* omega, int omega_rows, int omega_ld,
                             int oversample, int power, double eta, double floor_rel, int* counters,
                             void* stream) {
  if (n_bits < 1 || n_bits > 10 || batch < 0 || nterms < 1 || nterms > TN_MAXT || !terms || !dst ||
      !dst_ranks || chi_max < 1 || chi_max > dst_cap || chi_max > 512 || eps < 0 || !targets || !omega ||
      omega_rows < 1 || omega_ld < 1 || oversample < 0 || power < 0 || power > 4 || !(eta > 0.0) ||
      !(eta < 1.0) || floor_rel < 0.0 ||
      (precision != TNLBM_FP64 && precision != TNLBM_FP32)) {
    set_error("bad arguments to tnlbm_lincomb_round_rsvd");
    return TNLBM_E_ARG;
  }
  if (counters) counters[0] = counters[1] = counters[2] = 0;
  if (batch == 0) return 0;
  for (int i = 0; i < batch * (3 * n_bits + 1); ++i)
    if (targets[i] < 0) { set_error("negative target rank"); return TNLBM_E_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  tn::RsvdArgs ra{targets, omega, omega_rows, omega_ld, oversample, power, eta, floor_rel, counters};
  return precision == TNLBM_FP64
             ? tn::lincomb_impl<double>(n_bits, batch, nterms, terms, dst, dst_ranks, dst_cap, chi_max, eps, 0, st, &ra)
             : tn::lincomb_impl<float>(n_bits, batch, nterms, terms, dst, dst_ranks, dst_cap, chi_max, eps, 0, st, &ra);
}

int tnlbm_materialize(int precision, int n_bits, int batch, const tnlbm_term* terms, void* const* dst,
                      int* const* dst_ranks, int dst_cap, void* stream) {
  if (n_bits < 1 || n_bits > 10 || batch < 0 || !terms || !dst || !dst_ranks || dst_cap < 1) {
    set_error("bad arguments to tnlbm_materialize");
    return TNLBM_E_ARG;
  }
  if (batch == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == TNLBM_FP64
             ? tn::lincomb_impl<double>(n_bits, batch, 1, terms, dst, dst_ranks, dst_cap, 1, 0.0, 1, st)
             : tn::lincomb_impl<float>(n_bits, batch, 1, terms, dst, dst_ranks, dst_cap, 1, 0.0, 1, st);
}

int tnlbm_hadamard_zipup(int precision, int n_bits, int batch, const void* const* B, const int* const* rB,
                         int capB, const void* const* C, const int* const* rC, int capC, void* const* A,
                         int* const* rA, int capA, int chi_max, double eps, void* stream) {
  if (n_bits < 1 || n_bits > 10 || batch < 0 || !B || !rB || !C || !rC || !A || !rA || capB < 1 || capC < 1 ||
      capB > 512 || capC > 512 || chi_max < 1 || chi_max > 512 || capA < chi_max || eps < 0) {
    set_error("bad arguments to tnlbm_hadamard_zipup");
    return TNLBM_E_ARG;
  }
  if (batch == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == TNLBM_FP64
             ? tn::zipup_impl<double>(n_bits, batch, B, rB, capB, C, rC, capC, A, rA, capA, chi_max, eps, st)
             : tn::zipup_impl<float>(n_bits, batch, B, rB, capB, C, rC, capC, A, rA, capA, chi_max, eps, st);
}

int tnlbm_hadamard_fit(int precision, int n_bits, int batch, const void* const* B, const int* const* rB,
                       int capB, const void* const* C, const int* const* rC, int capC, void* const* A,
                       int* const* rA, int capA, int sweeps, void* stream) {
  if (n_bits < 1 || n_bits > 10 || batch < 0 || !B || !rB || !C || !rC || !A || !rA || capA < capB ||
      capB < 1 || capC < 1 || sweeps < 1 || capA > 1024 || capB * 2 > 1024) {
    set_error("bad arguments to tnlbm_hadamard_fit");
    return TNLBM_E_ARG;
  }
  if (batch == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == TNLBM_FP64
             ? tn::fit_impl<double>(n_bits, batch, false, B, rB, capB, C, rC, capC, A, rA, capA, sweeps, st)
             : tn::fit_impl<float>(n_bits, batch, prec_tc(precision), B, rB, capB, C, rC, capC, A, rA, capA,
                                   sweeps, st);
}

int tnlbm_inner_ones(int precision, int n_bits, int batch, const void* const* X, const int* const* rX,
                     int capX, double* out, void* stream) {
  if (n_bits < 1 || n_bits > 10 || batch < 0 || !X || !rX || !out || capX < 1 || capX > 1024) {
    set_error("bad arguments to tnlbm_inner_ones");
    return TNLBM_E_ARG;
  }
  if (batch == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<tn::MpsRef> refs(batch);
  for (int b = 0; b < batch; ++b) { refs[b].base = (void*)X[b]; refs[b].ranks = (int*)rX[b]; refs[b].cap = capX; }
  tn::DevBuf d;
  if (!d.alloc(batch * sizeof(tn::MpsRef))) { set_error("out of device memory"); return TNLBM_E_OOM; }
  TN_CUDA(cudaMemcpyAsync(d.p, refs.data(), batch * sizeof(tn::MpsRef), cudaMemcpyHostToDevice, st));
  if (precision == TNLBM_FP64) tn::launch_inner_ones<double>((const tn::MpsRef*)d.p, batch, 3 * n_bits, out, st);
  else tn::launch_inner_ones<float>((const tn::MpsRef*)d.p, batch, 3 * n_bits, out, st);
  TN_CUDA(cudaGetLastError());
  TN_CUDA(cudaStreamSynchronize(st));
  return 0;
}

int tnlbm_to_dense(int precision, int n_bits, const void* X, const int* rX, int capX, void* dense, void* stream) {
  if (n_bits < 1 || n_bits > 10 || !X || !rX || !dense || capX < 1 || capX > 1024) {
    set_error("bad arguments to tnlbm_to_dense");
    return TNLBM_E_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  tn::MpsRef m{(void*)X, (int*)rX, capX};
  const size_t es = precision == TNLBM_FP64 ? 8 : 4;
  const size_t sb = tn::contract_scratch_bytes(n_bits, capX, es);
  tn::DevBuf scr;
  if (!scr.alloc(sb)) { set_error("out of device memory"); return TNLBM_E_OOM; }
  int rc = precision == TNLBM_FP64 ? tn::contract_dense<double>(m, n_bits, (double*)dense, scr.p, sb, st)
                                   : tn::contract_dense<float>(m, n_bits, (float*)dense, scr.p, sb, st);
  if (rc) return rc;
  TN_CUDA(cudaGetLastError());
  TN_CUDA(cudaStreamSynchronize(st));
  return 0;
}

int tnlbm_from_dense(int precision, int n_bits, const void* dense, void* dst, int* dst_ranks, int dst_cap,
                     int chi_max, double eps, void* stream) {
  if (n_bits < 1 || n_bits > 10 || !dense || !dst || !dst_ranks || dst_cap < 1 || chi_max < 1 ||
      chi_max > dst_cap || 2 * chi_max > 1024 || eps < 0) {
    set_error("bad arguments to tnlbm_from_dense");
    return TNLBM_E_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  tn::DevBuf ds;
  if (!ds.alloc(STATUS_INTS * sizeof(int))) { set_error("out of device memory"); return TNLBM_E_OOM; }
  TN_CUDA(cudaMemsetAsync(ds.p, 0, STATUS_INTS * sizeof(int), st));
  int rc = precision == TNLBM_FP64
               ? tn::tt_svd_dense<double>((const double*)dense, n_bits, (double*)dst, dst_ranks, dst_cap, chi_max, eps, (int*)ds.p, st)
               : tn::tt_svd_dense<float>((const float*)dense, n_bits, (float*)dst, dst_ranks, dst_cap, chi_max, eps, (int*)ds.p, st);
  if (rc) return rc;
  return tn::check_status((int*)ds.p, st);
}

}  // extern "C"

// ================================================================ measurement
template <typename T>
static int profile_impl(tnlbm_sim* s, double* ms, double* flops, int* launches, double* phases) {
  using namespace tn;
  double* d_ctr = nullptr;
  TN_CUDA(cudaMalloc(&d_ctr, CTR_SIZE * sizeof(double)));
  cudaMemsetAsync(d_ctr, 0, CTR_SIZE * sizeof(double), s->s0);
  Prof prof;
  prof.st = s->s0;
  prof.d_ctr = d_ctr;
  prof.begin();
  int n = 0;
  enqueue_step<T>(s, &n, &prof);
  cudaError_t e = cudaStreamSynchronize(s->s0);
  if (e != cudaSuccess) { cudaFree(d_ctr); return cuda_fail(e, "tnlbm_profile_step"); }
  for (int c = 0; c < C_COUNT; ++c) { ms[c] = 0.0; launches[c] = 0; }
  prof.collect(ms, launches);
  double h_ctr[CTR_SIZE];
  cudaMemcpy(h_ctr, d_ctr, sizeof(h_ctr), cudaMemcpyDeviceToHost);
  for (int c = 0; c < C_COUNT; ++c) flops[c] = h_ctr[c];
  if (phases)
    for (int p = 0; p < PH_COUNT; ++p) phases[p] = h_ctr[C_COUNT + p];
  cudaFree(d_ctr);
  s->steps += 1;
  int st[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpy(st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[0]) { cudaMemset(s->d_status, 0, sizeof(st)); return status_to_code(st); }
  return 0;
}

extern "C" {

int tnlbm_step_timed(tnlbm_sim* s, int k, double* ms) {
  if (!s || k < 0 || !ms) { set_error("bad arguments to tnlbm_step_timed"); return TNLBM_E_ARG; }
  cudaEvent_t a, b;
  TN_CUDA(cudaEventCreate(&a));
  TN_CUDA(cudaEventCreate(&b));
  TN_CUDA(cudaEventRecord(a, s->s0));
  for (int i = 0; i < k; ++i) TN_CUDA(cudaGraphLaunch(s->gexec, s->s0));
  TN_CUDA(cudaEventRecord(b, s->s0));
  TN_CUDA(cudaEventSynchronize(b));
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t;
  s->steps += k;
  int st[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpy(st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[0]) { cudaMemset(s->d_status, 0, sizeof(st)); return status_to_code(st); }
  return 0;
}

int tnlbm_profile_step(tnlbm_sim* s, double* ms, double* flops, int* launches, double* phases) {
  if (!s || !ms || !flops || !launches) { set_error("bad arguments to tnlbm_profile_step"); return TNLBM_E_ARG; }
  return s->prec == TNLBM_FP64 ? profile_impl<double>(s, ms, flops, launches, phases)
                               : profile_impl<float>(s, ms, flops, launches, phases);
}

}  // extern "C"

// ================================================================ batched simulations
// Several independent simulations of the same lattice size stepped together:
// level l of the step launches the roundings and fits of level l of every
// simulation at once (each job carries its own simulation's masks, scalars and
// scratch), so that a launch holds the jobs of all of them.
struct tnlbm_batch {
  std::vector<tnlbm_sim*> sims;
  int prec = 0, sweeps = 2;
  Arena arena;
  cudaStream_t s0 = nullptr;
  std::vector<cudaStream_t> sfit;  // one fit stream per chain length in the batch
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<int> lens;           // distinct chain lengths L, ascending
  struct FitGroup {                // the fit and zip-up jobs of one chain length
    std::vector<FitJob> fj;
    FitJob* d_fj = nullptr;
    std::vector<ZipJob> zj;
    ZipJob* d_zj = nullptr;
  };
  struct Level {
    std::vector<RoundJob> rj;      // all simulations' rounding jobs (each carries its L)
    std::vector<FitGroup> fg;      // indexed like lens
    RoundJob* d_rj = nullptr;
    std::vector<int> rho0;         // simulations with a rho_0 node at this level
    int cluster = 1;               // CTAs per rounding job of this level
  };
  std::vector<Level> levels;
  int* d_status = nullptr;
  struct CopyGroup {
    MpsRef* d_src = nullptr;
    MpsRef* d_dst = nullptr;
    int n = 0;
  };
  std::vector<CopyGroup> copies;   // indexed like lens
  int launches_per_step = 0;
  int cap = 16;                    // largest cluster size (smallest max_cluster of the simulations)
};

namespace tn {

template <typename T>
static int enqueue_batch_step(tnlbm_batch* b, int* launches) {
  int nl = 0;
  const int ng = (int)b->lens.size();
  for (auto& lv : b->levels) {
    for (int si : lv.rho0) {
      tnlbm_sim* s = b->sims[si];
      launch_rho0<T>(s->d_rho_ref, s->L, s->n_fluid, s->d_scal, b->s0);
      ++nl;
    }
    bool any_fit = false;
    for (auto& g : lv.fg) any_fit = any_fit || !g.fj.empty() || !g.zj.empty();
    // fits of each chain length on their own stream, beside the level's roundings
    if (any_fit) {
      cudaEventRecord(b->ev_fork, b->s0);
      for (int gi = 0; gi < ng; ++gi)
        if (!lv.fg[gi].fj.empty() || !lv.fg[gi].zj.empty()) cudaStreamWaitEvent(b->sfit[gi], b->ev_fork, 0);
      for (int gi = 0; gi < ng; ++gi) {
        auto& g = lv.fg[gi];
        if (!g.fj.empty())
          nl += run_fit<T>(g.d_fj, g.fj, b->lens[gi], b->sweeps, b->d_status, b->sfit[gi], nullptr,
                           prec_tc(b->prec));
        if (!g.zj.empty())
          nl += run_zipup<T>(g.d_zj, (int)g.zj.size(), b->lens[gi], b->d_status, b->sfit[gi], nullptr);
      }
    }
    if (!lv.rj.empty()) {
      launch_round<T>(lv.d_rj, (int)lv.rj.size(), b->lens.back(), 0, nullptr, nullptr, b->d_status, b->s0,
                      nullptr, nullptr, lv.cluster);
      ++nl;
    }
    if (any_fit)
      for (int gi = 0; gi < ng; ++gi) {
        if (lv.fg[gi].fj.empty() && lv.fg[gi].zj.empty()) continue;
        cudaEventRecord(b->ev_join[gi], b->sfit[gi]);
        cudaStreamWaitEvent(b->s0, b->ev_join[gi], 0);
      }
  }
  for (tnlbm_sim* s : b->sims)
    if (s->cfg.conserve_mass) {
      launch_mass_fix<T>(s->d_copy_src, s->lat.Q, s->L, s->d_mass, s->d_mass0, b->s0);
      nl += 2;
    }
  for (int gi = 0; gi < ng; ++gi) {
    launch_copy<T>(b->copies[gi].d_src, b->copies[gi].d_dst, b->copies[gi].n, b->lens[gi], b->s0);
    ++nl;
  }
  *launches = nl;
  return 0;
}

// (re)capture one batched step as a graph
template <typename T>
static int batch_capture(tnlbm_batch* b) {
  TN_CUDA(cudaStreamSynchronize(b->s0));
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  TN_CUDA(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal));
  int launches = 0;
  enqueue_batch_step<T>(b, &launches);
  TN_CUDA(cudaStreamEndCapture(b->s0, &b->graph));
  TN_CUDA(cudaGraphInstantiate(&b->gexec, b->graph, 0));
  b->launches_per_step = launches;
  return 0;
}

// tune_sim for a batch: one eager batched step on s0 without the final
// copies, each level's rounding launch timed at the candidate cluster sizes.
template <typename T>
static int tune_batch(tnlbm_batch* b, int reps, double* ms, int ms_cap) {
  for (tnlbm_sim* s : b->sims)
    if (s->learn_mode) { set_error("tune the cluster sizes before configuring the learned rounding"); return TNLBM_E_ARG; }
  TN_CUDA(cudaStreamSynchronize(b->s0));
  const int ns = (int)b->sims.size();
  std::vector<double> disc(ns, 0.0);
  for (int i = 0; i < ns; ++i)
    TN_CUDA(cudaMemcpy(&disc[i], b->sims[i]->d_discard, sizeof(double), cudaMemcpyDeviceToHost));
  const bool tune = clusters_apply(b->prec) && b->cap > 1;
  std::vector<int> old;
  for (auto& lv : b->levels) old.push_back(lv.cluster);
  std::vector<double> t((size_t)b->levels.size() * (TNLBM_CLUSTER_MAX + 1), -1.0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TN_CUDA(cudaEventCreate(&e0));
  TN_CUDA(cudaEventCreate(&e1));
  int rc = 0;
  for (size_t l = 0; l < b->levels.size() && !rc; ++l) {
    auto& lv = b->levels[l];
    for (int si : lv.rho0) {
      tnlbm_sim* s = b->sims[si];
      launch_rho0<T>(s->d_rho_ref, s->L, s->n_fluid, s->d_scal, b->s0);
    }
    for (size_t gi = 0; gi < b->lens.size(); ++gi) {
      auto& g = lv.fg[gi];
      if (!g.fj.empty())
        run_fit<T>(g.d_fj, g.fj, b->lens[gi], b->sweeps, b->d_status, b->s0, nullptr, prec_tc(b->prec));
      if (!g.zj.empty()) run_zipup<T>(g.d_zj, (int)g.zj.size(), b->lens[gi], b->d_status, b->s0, nullptr);
    }
    if (lv.rj.empty()) continue;
    auto run = [&](int P) {
      launch_round<T>(lv.d_rj, (int)lv.rj.size(), b->lens.back(), 0, nullptr, nullptr, b->d_status, b->s0,
                      nullptr, nullptr, P);
    };
    if (tune) {
      int best = lv.cluster;
      rc = tune_launch<T>(run, b->cap, reps, lv.cluster, b->s0, e0, e1,
                          t.data() + l * (TNLBM_CLUSTER_MAX + 1), &best);
      if (!rc) lv.cluster = best;
    } else {
      run(lv.cluster);
    }
  }
  cudaStreamSynchronize(b->s0);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < ns; ++i)
    TN_CUDA(cudaMemcpy(b->sims[i]->d_discard, &disc[i], sizeof(double), cudaMemcpyHostToDevice));
  int st[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpy(st, b->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (!rc && st[0]) {
    rc = status_to_code(st);
    TN_CUDA(cudaMemset(b->d_status, 0, STATUS_INTS * sizeof(int)));
  }
  if (rc)
    for (size_t l = 0; l < b->levels.size(); ++l) b->levels[l].cluster = old[l];
  else if (ms)
    std::copy(t.begin(), t.begin() + std::min<size_t>(t.size(), std::max(ms_cap, 0)), ms);
  const int rc2 = batch_capture<T>(b);
  return rc ? rc : rc2;
}

template <typename T>
static int batch_build(tnlbm_batch* b) {
  for (tnlbm_sim* s : b->sims) b->lens.push_back(s->L);
  std::sort(b->lens.begin(), b->lens.end());
  b->lens.erase(std::unique(b->lens.begin(), b->lens.end()), b->lens.end());
  const int ng = (int)b->lens.size();
  for (tnlbm_sim* s : b->sims) b->cap = std::min(b->cap, s->cfg.max_cluster > 0 ? s->cfg.max_cluster : 16);
  auto group = [&](int L) { return (int)(std::lower_bound(b->lens.begin(), b->lens.end(), L) - b->lens.begin()); };
  TN_CUDA(cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking));
  TN_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  b->sfit.assign(ng, nullptr);
  b->ev_join.assign(ng, nullptr);
  for (int gi = 0; gi < ng; ++gi) {
    TN_CUDA(cudaStreamCreateWithFlags(&b->sfit[gi], cudaStreamNonBlocking));
    TN_CUDA(cudaEventCreateWithFlags(&b->ev_join[gi], cudaEventDisableTiming));
  }
  b->d_status = (int*)b->arena.alloc(STATUS_INTS * sizeof(int));
  if (!b->d_status) return TNLBM_E_OOM;
  TN_CUDA(cudaMemset(b->d_status, 0, STATUS_INTS * sizeof(int)));
  size_t nlev = 0;
  for (tnlbm_sim* s : b->sims) nlev = std::max(nlev, s->levels.size());
  tnlbm_batch::Level empty;
  empty.fg.resize(ng);
  b->levels.assign(nlev, empty);
  std::vector<std::vector<MpsRef>> src(ng), dst(ng);
  for (int si = 0; si < (int)b->sims.size(); ++si) {
    tnlbm_sim* s = b->sims[si];
    const int gi = group(s->L);
    for (size_t l = 0; l < s->levels.size(); ++l) {
      auto& in = s->levels[l];
      auto& out = b->levels[l];
      for (RoundJob rj : in.rj) {
        rj.masks = s->d_masks;
        rj.scal = s->d_scal;
        rj.L = s->L;
        rj.n_bits = s->n;
        out.rj.push_back(rj);
      }
      for (const FitJob& fj : in.fj) out.fg[gi].fj.push_back(fj);
      for (const ZipJob& zj : in.zj) out.fg[gi].zj.push_back(zj);
      if (in.has_rho0) out.rho0.push_back(si);
    }
    for (int i = 0; i < s->lat.Q; ++i) {
      src[gi].push_back(s->nodes[s->f_next[i]]);
      dst[gi].push_back(s->nodes[s->f_state[i]]);
    }
  }
  for (auto& lv : b->levels) {
    if (!lv.rj.empty()) {
      lv.d_rj = (RoundJob*)b->arena.alloc(lv.rj.size() * sizeof(RoundJob));
      if (!lv.d_rj) return TNLBM_E_OOM;
      TN_CUDA(cudaMemcpy(lv.d_rj, lv.rj.data(), lv.rj.size() * sizeof(RoundJob), cudaMemcpyHostToDevice));
      lv.cluster = clusters_apply(b->prec) && b->cap > 1 ? round_cluster_size<T>((int)lv.rj.size(), b->cap) : 1;
    }
    for (auto& g : lv.fg) {
      if (g.fj.empty()) continue;
      g.d_fj = (FitJob*)b->arena.alloc(g.fj.size() * sizeof(FitJob));
      if (!g.d_fj) return TNLBM_E_OOM;
      TN_CUDA(cudaMemcpy(g.d_fj, g.fj.data(), g.fj.size() * sizeof(FitJob), cudaMemcpyHostToDevice));
    }
    for (auto& g : lv.fg) {
      if (g.zj.empty()) continue;
      g.d_zj = (ZipJob*)b->arena.alloc(g.zj.size() * sizeof(ZipJob));
      if (!g.d_zj) return TNLBM_E_OOM;
      TN_CUDA(cudaMemcpy(g.d_zj, g.zj.data(), g.zj.size() * sizeof(ZipJob), cudaMemcpyHostToDevice));
    }
  }
  b->copies.assign(ng, tnlbm_batch::CopyGroup{});
  for (int gi = 0; gi < ng; ++gi) {
    auto& c = b->copies[gi];
    c.n = (int)src[gi].size();
    c.d_src = (MpsRef*)b->arena.alloc(c.n * sizeof(MpsRef));
    c.d_dst = (MpsRef*)b->arena.alloc(c.n * sizeof(MpsRef));
    if (!c.d_src || !c.d_dst) return TNLBM_E_OOM;
    TN_CUDA(cudaMemcpy(c.d_src, src[gi].data(), c.n * sizeof(MpsRef), cudaMemcpyHostToDevice));
    TN_CUDA(cudaMemcpy(c.d_dst, dst[gi].data(), c.n * sizeof(MpsRef), cudaMemcpyHostToDevice));
  }
  TN_CUDA(cudaDeviceSynchronize());
  return batch_capture<T>(b);
}

static int batch_status(tnlbm_batch* b) {
  int st[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpy(st, b->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[0]) {
    cudaMemset(b->d_status, 0, sizeof(st));
    return status_to_code(st);
  }
  return 0;
}

}  // namespace tn

extern "C" {

int tnlbm_batch_destroy(tnlbm_batch* b) {
  if (!b) return 0;
  if (b->s0) cudaStreamSynchronize(b->s0);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  if (b->s0) cudaStreamDestroy(b->s0);
  for (cudaStream_t st : b->sfit)
    if (st) cudaStreamDestroy(st);
  for (tnlbm_sim* s : b->sims) tnlbm_destroy(s);
  delete b;
  return 0;
}

int tnlbm_batch_create(const tnlbm_config* cfgs, int nsim, tnlbm_batch** out) {
  if (!out) { set_error("out is NULL"); return TNLBM_E_ARG; }
  *out = nullptr;
  if (!cfgs || nsim < 1 || nsim > 64) { set_error("bad arguments to tnlbm_batch_create"); return TNLBM_E_ARG; }
  for (int i = 1; i < nsim; ++i)
    if (cfgs[i].precision != cfgs[0].precision || std::max(cfgs[i].sweeps, 0) != std::max(cfgs[0].sweeps, 0)) {
      set_error("batched simulations need the same precision and fit sweeps");
      return TNLBM_E_ARG;
    }
  // the batched rounding launches carry no learned-rounding context: a
  // simulation with the learned rounding is stepped alone
  for (int i = 0; i < nsim; ++i)
    if (cfgs[i].learned_rank != 0) {
      set_error("batched simulations take the full SVD: learned_rank must be 0 (step such a simulation alone)");
      return TNLBM_E_ARG;
    }
  tnlbm_batch* b = new (std::nothrow) tnlbm_batch();
  if (!b) { set_error("host allocation failed"); return TNLBM_E_OOM; }
  for (int i = 0; i < nsim; ++i) {
    tnlbm_sim* s = nullptr;
    int rc = tnlbm_create(&cfgs[i], &s);
    if (rc) {
      std::string msg = tn::g_err;
      tnlbm_batch_destroy(b);
      tn::g_err = "simulation " + std::to_string(i) + " of the batch: " + msg;
      return rc;
    }
    b->sims.push_back(s);
  }
  b->prec = b->sims[0]->prec;
  b->sweeps = b->sims[0]->cfg.sweeps;
  int rc = b->prec == TNLBM_FP64 ? tn::batch_build<double>(b) : tn::batch_build<float>(b);
  if (rc) {
    std::string msg = tn::g_err;
    tnlbm_batch_destroy(b);
    tn::g_err = msg;
    return rc;
  }
  *out = b;
  return 0;
}

int tnlbm_batch_step(tnlbm_batch* b, int k) {
  if (!b || k < 0) { set_error("bad arguments to tnlbm_batch_step"); return TNLBM_E_ARG; }
  for (int i = 0; i < k; ++i) TN_CUDA(cudaGraphLaunch(b->gexec, b->s0));
  TN_CUDA(cudaStreamSynchronize(b->s0));
  for (tnlbm_sim* s : b->sims) s->steps += k;
  return tn::batch_status(b);
}

int tnlbm_batch_step_timed(tnlbm_batch* b, int k, double* ms) {
  if (!b || k < 0 || !ms) { set_error("bad arguments to tnlbm_batch_step_timed"); return TNLBM_E_ARG; }
  cudaEvent_t e0, e1;
  TN_CUDA(cudaEventCreate(&e0));
  TN_CUDA(cudaEventCreate(&e1));
  TN_CUDA(cudaEventRecord(e0, b->s0));
  for (int i = 0; i < k; ++i) TN_CUDA(cudaGraphLaunch(b->gexec, b->s0));
  TN_CUDA(cudaEventRecord(e1, b->s0));
  TN_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t;
  for (tnlbm_sim* s : b->sims) s->steps += k;
  return tn::batch_status(b);
}

tnlbm_sim* tnlbm_batch_sim(tnlbm_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->sims.size()) { set_error("bad arguments to tnlbm_batch_sim"); return nullptr; }
  return b->sims[i];
}

int tnlbm_batch_info(tnlbm_batch* b, int* nsim, int* launches_per_step, int* jobs_per_step) {
  if (!b) { set_error("bad arguments to tnlbm_batch_info"); return TNLBM_E_ARG; }
  if (nsim) *nsim = (int)b->sims.size();
  if (launches_per_step) *launches_per_step = b->launches_per_step;
  if (jobs_per_step) {
    int j = 0;
    for (auto& lv : b->levels) {
      j += (int)lv.rj.size();
      for (auto& g : lv.fg) j += (int)(g.fj.size() + g.zj.size());
    }
    *jobs_per_step = j;
  }
  return 0;
}

int tnlbm_batch_clusters(tnlbm_batch* b, int* clusters, int* jobs, int cap, int* nlevels) {
  if (!b) { set_error("bad arguments to tnlbm_batch_clusters"); return TNLBM_E_ARG; }
  return tn::get_clusters(b->levels, clusters, jobs, cap, nlevels);
}

int tnlbm_batch_set_clusters(tnlbm_batch* b, const int* clusters, int nlevels) {
  if (!b) { set_error("bad arguments to tnlbm_batch_set_clusters"); return TNLBM_E_ARG; }
  const bool f64 = b->prec == TNLBM_FP64;
  int rc = f64 ? tn::set_clusters<double>(b->levels, b->prec, clusters, nlevels)
               : tn::set_clusters<float>(b->levels, b->prec, clusters, nlevels);
  if (rc) return rc;
  return f64 ? tn::batch_capture<double>(b) : tn::batch_capture<float>(b);
}

int tnlbm_batch_tune_clusters(tnlbm_batch* b, int reps, double* ms, int ms_cap) {
  if (!b || reps < 1 || (ms && ms_cap < 0)) { set_error("bad arguments to tnlbm_batch_tune_clusters"); return TNLBM_E_ARG; }
  return b->prec == TNLBM_FP64 ? tn::tune_batch<double>(b, reps, ms, ms_cap) : tn::tune_batch<float>(b, reps, ms, ms_cap);
}

}  // extern "C"
