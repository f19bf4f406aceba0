// pc_model.cpp -- market model setup on the host: validation, Cholesky
// factor of the correlation, breadth-first Brownian-bridge schedule arranged
// in date order, and the drift / discount / static-value tables.
//
// The paper leaves the pricing engine's model open (Sec. 6.2 names an MC
// engine without details).  The engine simulates a correlated Black-Scholes
// market on the model's date grid:
//   W: Brownian motions at the grid dates, built by breadth-first bisection;
//   X = L W with L the Cholesky factor of the correlation matrix;
//   S_l(o) = S0_l exp((r - sigma_l^2 / 2) tau_o + sigma_l X_l(o)),
//   tau_o = day_o / 365; discount d(o) = exp(-r tau_o).
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <utility>

#include "pc_internal.h"

namespace pc {

namespace {

bool finite(double x) { return std::isfinite(x); }

// FP64 Cholesky factor L (row-major, lower) of the d x d matrix c; false if
// c is not symmetric positive definite.
bool cholesky(int d, const std::vector<double> &c, std::vector<double> &L) {
  L.assign(size_t(d) * d, 0.0);
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = c[size_t(i) * d + j];
      for (int k = 0; k < j; ++k) s -= L[size_t(i) * d + k] * L[size_t(j) * d + k];
      if (i == j) {
        if (!(s > 1e-12)) return false;
        L[size_t(i) * d + i] = std::sqrt(s);
      } else {
        L[size_t(i) * d + j] = s / L[size_t(j) * d + j];
      }
    }
  }
  return true;
}

struct Node {
  int m, l, r, level;
  double wl, wr, sd;
};

}  // namespace

pc_status build_model(const pc_model_desc &desc, ModelHost &M, std::string &err) {
  const int d = desc.d, n = desc.n_dates, H = desc.n_hist;
  if (d < 1 || d > PC_MAX_UNDERLYINGS) {
    err = "d must be in 1..4";
    return d > PC_MAX_UNDERLYINGS ? PC_ELIMIT : PC_EINVAL;
  }
  if (n < 1) { err = "n_dates must be >= 1"; return PC_EINVAL; }
  if (n > PC_MAX_DATES) { err = "n_dates exceeds PC_MAX_DATES"; return PC_ELIMIT; }
  if (H < 0) { err = "n_hist must be >= 0"; return PC_EINVAL; }
  if (H > PC_MAX_HISTORY) { err = "n_hist exceeds PC_MAX_HISTORY"; return PC_ELIMIT; }
  if (!desc.S0 || !desc.sigma || !desc.corr || !desc.day) { err = "null model array"; return PC_EINVAL; }
  if (H > 0 && (!desc.history || !desc.hist_day)) { err = "null history array"; return PC_EINVAL; }
  if (desc.t_now < 0) { err = "t_now must be >= 0"; return PC_EINVAL; }
  if (!finite(desc.r)) { err = "r not finite"; return PC_EINVAL; }
  for (int i = 0; i < d; ++i) {
    if (!(desc.S0[i] > 0) || !finite(desc.S0[i])) { err = "S0 must be finite and > 0"; return PC_EINVAL; }
    if (!(desc.sigma[i] >= 0) || !finite(desc.sigma[i])) { err = "sigma must be finite and >= 0"; return PC_EINVAL; }
  }
  for (int k = 0; k < n; ++k) {
    if (desc.day[k] <= 0 || (k && desc.day[k] <= desc.day[k - 1])) {
      err = "day[] must be > 0 and strictly increasing";
      return PC_EINVAL;
    }
  }
  for (int k = 0; k < H; ++k) {
    if (desc.hist_day[k] >= 0 || (k && desc.hist_day[k] >= desc.hist_day[k - 1])) {
      err = "hist_day[] must be < 0 and strictly decreasing";
      return PC_EINVAL;
    }
    for (int l = 0; l < d; ++l)
      if (!finite(desc.history[size_t(k) * d + l])) { err = "history not finite"; return PC_EINVAL; }
  }
  M.d = d; M.n = n; M.n_hist = H; M.t_now = desc.t_now; M.r = desc.r;
  M.S0.assign(desc.S0, desc.S0 + d);
  M.sigma.assign(desc.sigma, desc.sigma + d);
  M.corr.assign(desc.corr, desc.corr + size_t(d) * d);
  M.day.assign(desc.day, desc.day + n);
  if (H) {
    M.hist_day.assign(desc.hist_day, desc.hist_day + H);
    M.history.assign(desc.history, desc.history + size_t(H) * d);
  }
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j < d; ++j) {
      double a = M.corr[size_t(i) * d + j], b = M.corr[size_t(j) * d + i];
      if (!finite(a) || std::fabs(a - b) > 1e-12 || (i == j && std::fabs(a - 1.0) > 1e-12)) {
        err = "corr must be symmetric with unit diagonal";
        return PC_ENOTPD;
      }
    }
  }
  if (!cholesky(d, M.corr, M.L)) { err = "corr is not positive definite"; return PC_ENOTPD; }

  // Year fractions of ordinals 0..n.
  std::vector<double> tau(n + 1, 0.0);
  for (int o = 1; o <= n; ++o) tau[o] = M.day[o - 1] / 365.0;

  // Breadth-first bisection nodes: node 0 is date n; then intervals from a
  // FIFO starting at (0, n), each of length >= 2 producing its midpoint.
  std::vector<Node> nodes;
  std::map<std::pair<int, int>, int> node_of;  // interval (l, r) -> node
  nodes.push_back({n, 0, -1, 0, 0.0, 0.0, std::sqrt(tau[n])});
  std::deque<std::pair<std::pair<int, int>, int>> q;  // ((l, r), level of its node)
  q.push_back({{0, n}, 1});
  while (!q.empty()) {
    auto [lr, lev] = q.front();
    q.pop_front();
    auto [l, r] = lr;
    if (r - l < 2) continue;
    int m = (l + r) / 2;
    double span = tau[r] - tau[l];
    node_of[{l, r}] = int(nodes.size());
    nodes.push_back({m, l, r, lev, (tau[r] - tau[m]) / span, (tau[m] - tau[l]) / span,
                     std::sqrt((tau[m] - tau[l]) * (tau[r] - tau[m]) / span)});
    q.push_back({{l, m}, lev + 1});
    q.push_back({{m, r}, lev + 1});
  }
  int n_levels = 0;
  for (auto &nd : nodes) n_levels = std::max(n_levels, nd.level + 1);

  // Date-order schedule (see BridgeOp in pc_types.h).
  M.date_ops.assign(n + 2, 0);
  M.ops.clear();
  std::vector<int> stk;  // dates whose W is computed but not yet produced
  int cur = 0, depth_max = 0;
  for (int t = 1; t <= n; ++t) {
    M.date_ops[t] = int(M.ops.size());
    std::vector<int> js;
    if (t == 1) {
      js.push_back(0);
      stk.push_back(n);
    }
    while (stk.back() != t) {
      auto it = node_of.find({cur, stk.back()});
      if (it == node_of.end()) { err = "internal: bridge schedule"; return PC_EINVAL; }
      js.push_back(it->second);
      stk.push_back(nodes[it->second].m);
    }
    // the kernel pushes every op's node and then pops the date's value, so
    // it holds the schedule's stack including the date itself
    depth_max = std::max(depth_max, int(stk.size()));
    stk.pop_back();
    cur = t;
    for (int j : js) {
      BridgeOp op{};
      const Node &nd = nodes[j];
      op.wl = op.wl_ = float(nd.wl);
      op.wr = op.wr_ = float(nd.wr);
      op.sd = op.sd_ = float(nd.sd);
      op.j = uint32_t(j);
      op.m = uint16_t(nd.m);
      op.flags = nd.r < 0 ? BR_ROOT : 0;
      M.ops.push_back(op);  // op k takes normals d k .. d k + d - 1
    }
  }
  M.date_ops[n + 1] = int(M.ops.size());
  M.n_levels = n_levels;
  M.bstack = std::max(depth_max, 1);

  // Tables.
  const double log2e = 1.4426950408889634;
  M.A.assign(size_t(n + 1) * d, float2{0.f, 0.f});
  for (int o = 0; o <= n; ++o)
    for (int i = 0; i < d; ++i) {
      const float a = float(log2e * (M.r - 0.5 * M.sigma[i] * M.sigma[i]) * tau[o]);
      M.A[size_t(o) * d + i] = float2{a, a};
    }
  M.B.assign(size_t(d) * d, 0.f);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) M.B[size_t(i) * d + k] = float(log2e * M.sigma[i] * M.L[size_t(i) * d + k]);
  M.disc.assign(size_t(H + n + 1), 0.f);
  for (int o = -H; o <= n; ++o) {
    double day = o > 0 ? M.day[o - 1] : (o == 0 ? 0.0 : M.hist_day[-o - 1]);
    M.disc[size_t(o + H)] = float(std::exp(-M.r * day / 365.0));
  }
  M.sval.assign(size_t(H + 1) * d, 0.f);
  for (int o = -H; o <= 0; ++o)
    for (int l = 0; l < d; ++l)
      M.sval[size_t(o + H) * d + l] =
          float(o == 0 ? M.S0[l] : M.history[size_t(-o - 1) * d + l]);
  M.tau.assign(size_t(n + 1), 0.f);
  for (int o = 0; o <= n; ++o) M.tau[o] = float(tau[o]);
  M.Lf.assign(M.L.begin(), M.L.end());
  M.sig.assign(M.sigma.begin(), M.sigma.end());
  return PC_OK;
}

}  // namespace pc
