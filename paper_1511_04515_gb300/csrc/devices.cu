// The device list of the C ABI (ers_create / ers_create_batch take `devices, ndevices`).
//
// A single circuit does not shard: every G_k^-1 of Algorithm 1 couples all of its nodes, so a
// context lives on exactly one device and several devices give replicas (one context each).
// A batch of independent circuits shards with no exchange on the data path: its instances
// are split over the devices by longest-processing-time-first on an estimated cost, each
// device share becomes an ordinary batched context on that device, and the group context
// returned to the caller only dispatches -- per-instance results are gathered on the host in
// input order.  Shares on one device run one after the other; shares on different devices
// run concurrently, one host thread per device.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "controller.h"
#include "ers_internal.h"

namespace ers {

// LPT: instances by decreasing cost, each onto the least-loaded part (ties: lowest part).
// Bounds the largest load by (4/3 - 1/(3 nparts)) times the optimum (Graham 1969).
void lpt_partition(const double* cost, int n, int nparts, int32_t* part_of) {
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  using Slot = std::pair<double, int>;   // (load, part)
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  for (int p = 0; p < nparts; ++p) heap.push({0.0, p});
  for (int i : order) {
    Slot s = heap.top();
    heap.pop();
    part_of[i] = s.second;
    heap.push({s.first + cost[i], s.second});
  }
}

// Estimated cost of one instance: the pattern of G_k (linear part plus device stamps) and its
// node count, a proxy of its factor size; instances of one family take similar step counts.
double instance_cost(const ers_instance& I) {
  double nnz = I.G ? (double)I.G->nnz : 0.0;
  double n = I.G ? (double)I.G->n_rows : 0.0;
  return nnz + n + 6.0 * std::max(I.ndev, 0);
}

std::string check_device_list(const int32_t* devices, int32_t ndevices) {
  if (ndevices < 0) return "ndevices must be >= 0";
  if (ndevices == 0) return "";
  if (!devices) return "devices is NULL but ndevices > 0";
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return std::string("no CUDA device: ") + cudaGetErrorString(e);
  }
  for (int32_t i = 0; i < ndevices; ++i)
    if (devices[i] < 0 || devices[i] >= count)
      return "device " + std::to_string(devices[i]) + " does not exist (" +
             std::to_string(count) + " visible)";
  return "";
}

static ers_status group_fail(ers_ctx* g, ers_status st, const std::string& msg) {
  g->err = msg;
  return st;
}

// Run f(sub, index) on every sub-context with its device current: one host thread per
// distinct device, the shares of one device in order.  Returns the first failure.
template <class F>
static ers_status group_each(ers_ctx* g, F f) {
  std::vector<int> devs = g->group_dev;
  std::sort(devs.begin(), devs.end());
  devs.erase(std::unique(devs.begin(), devs.end()), devs.end());
  std::vector<ers_status> st(g->group.size(), ERS_OK);
  auto work = [&](int dev) {
    DeviceGuard dg(dev);
    for (size_t q = 0; q < g->group.size(); ++q)
      if (g->group_dev[q] == dev) st[q] = f(g->group[q], (int)q);
  };
  if (devs.size() == 1) {
    work(devs[0]);
  } else {
    std::vector<std::thread> th;
    for (int d : devs) th.emplace_back(work, d);
    for (auto& t : th) t.join();
  }
  for (size_t q = 0; q < g->group.size(); ++q)
    if (st[q] != ERS_OK)
      return group_fail(g, st[q], "device " + std::to_string(g->group_dev[q]) + " share " +
                                      std::to_string(q) + ": " + g->group[q]->err);
  return ERS_OK;
}

ers_status group_call(ers_ctx* g, const std::function<ers_status(ers_ctx*, int)>& f) {
  return group_each(g, f);
}

// concatenated vector of the whole batch (input order) <-> per-share concatenations
static void split_state(const ers_ctx* g, const double* x, std::vector<std::vector<double>>& xs) {
  xs.assign(g->group.size(), {});
  for (int k = 0; k < g->ninst; ++k) {
    auto& dst = xs[g->inst_grp[k]];
    dst.insert(dst.end(), x + g->inst_off[k], x + g->inst_off[k] + g->inst_n[k]);
  }
}

static void join_state(const ers_ctx* g, const std::vector<std::vector<double>>& xs, double* x) {
  std::vector<size_t> pos(g->group.size(), 0);
  for (int k = 0; k < g->ninst; ++k) {
    int q = g->inst_grp[k];
    std::memcpy(x + g->inst_off[k], xs[q].data() + pos[q], sizeof(double) * g->inst_n[k]);
    pos[q] += g->inst_n[k];
  }
}

ers_status group_create(ers_ctx* g, const ers_instance* inst, int32_t ninst,
                        const int32_t* devices, int32_t ndevices, const ers_opts* opts) {
  std::vector<double> cost(ninst);
  for (int k = 0; k < ninst; ++k) cost[k] = instance_cost(inst[k]);
  std::vector<int32_t> part(ninst);
  lpt_partition(cost.data(), ninst, ndevices, part.data());
  g->grouped = true;
  g->device = -1;
  g->ninst = ninst;
  g->inst_grp.assign(ninst, -1);
  g->inst_loc.assign(ninst, -1);
  g->inst_n.assign(ninst, 0);
  g->inst_off.assign(ninst + 1, 0);
  for (int k = 0; k < ninst; ++k) {
    g->inst_n[k] = inst[k].G ? inst[k].G->n_rows : 0;
    g->inst_off[k + 1] = g->inst_off[k] + g->inst_n[k];
  }
  g->n = g->inst_off[ninst];
  for (int p = 0; p < ndevices; ++p) {
    std::vector<ers_instance> mine;
    std::vector<int32_t> idx;
    for (int k = 0; k < ninst; ++k)
      if (part[k] == p) {
        idx.push_back(k);
        mine.push_back(inst[k]);
      }
    if (mine.empty()) continue;      // more devices than instances
    ers_ctx* sub = nullptr;
    ers_status st;
    {
      DeviceGuard dg(devices[p]);
      st = create_batch_here(&sub, mine.data(), (int32_t)mine.size(), opts);
    }
    if (st != ERS_OK) {
      std::string msg = sub ? sub->err : std::string("out of memory");
      if (sub) {
        DeviceGuard dg(devices[p]);
        ers_destroy(sub);
      }
      return group_fail(g, st, "device " + std::to_string(devices[p]) + ": " + msg);
    }
    const int q = (int)g->group.size();
    for (size_t a = 0; a < idx.size(); ++a) {
      g->inst_grp[idx[a]] = q;
      g->inst_loc[idx[a]] = (int32_t)a;
    }
    g->group.push_back(sub);
    g->group_dev.push_back(devices[p]);
    g->group_inst.push_back(idx);
  }
  g->device = -1;
  if (opts) g->opts = *opts; else ers_default_opts(&g->opts);
  return ERS_OK;
}

void group_destroy(ers_ctx* g) {
  for (size_t q = 0; q < g->group.size(); ++q) {
    DeviceGuard dg(g->group_dev[q]);
    ers_destroy(g->group[q]);
  }
  for (size_t q = 0; q < g->group_nets.size(); ++q) {
    if (!g->group_nets[q]) continue;
    DeviceGuard dg(g->group_dev[q]);
    ers_mlp_destroy(g->group_nets[q]);
  }
  g->group.clear();
  g->group_nets.clear();
}

ers_status group_run_batch(ers_ctx* g, double t_end, double tol, int32_t max_steps,
                           int32_t* nsteps, int32_t* nreject) {
  std::vector<std::vector<int32_t>> ns(g->group.size()), nr(g->group.size());
  for (size_t q = 0; q < g->group.size(); ++q) {
    ns[q].assign(g->group_inst[q].size(), 0);
    nr[q].assign(g->group_inst[q].size(), 0);
  }
  ers_status st = group_each(g, [&](ers_ctx* s, int q) {
    return ers_run_batch(s, t_end, tol, max_steps, ns[q].data(), nr[q].data());
  });
  for (int k = 0; k < g->ninst; ++k) {
    int q = g->inst_grp[k], l = g->inst_loc[k];
    if (nsteps) nsteps[k] = ns[q][l];
    if (nreject) nreject[k] = nr[q][l];
  }
  return st;
}

ers_status group_dc(ers_ctx* g, const double* x0) {
  std::vector<std::vector<double>> xs;
  if (x0) split_state(g, x0, xs);
  return group_each(g, [&](ers_ctx* s, int q) { return ers_dc(s, x0 ? xs[q].data() : nullptr); });
}

ers_status group_set_state(ers_ctx* g, double t, const double* x, double h) {
  std::vector<std::vector<double>> xs;
  split_state(g, x, xs);
  return group_each(g, [&](ers_ctx* s, int q) { return ers_set_state(s, t, xs[q].data(), h); });
}

ers_status group_get_state(ers_ctx* g, double* t, double* x, double* h) {
  std::vector<std::vector<double>> xs(g->group.size());
  for (size_t q = 0; q < g->group.size(); ++q) xs[q].assign(g->group[q]->n, 0.0);
  std::vector<double> ts(g->group.size()), hs(g->group.size());
  ers_status st = group_each(g, [&](ers_ctx* s, int q) {
    return ers_get_state(s, &ts[q], x ? xs[q].data() : nullptr, &hs[q]);
  });
  if (st != ERS_OK) return st;
  if (t) *t = ts.empty() ? 0.0 : *std::min_element(ts.begin(), ts.end());
  if (h) *h = hs.empty() ? 0.0 : hs[0];
  if (x) join_state(g, xs, x);
  return ERS_OK;
}

// b -> x for the block-diagonal matrix of the whole batch (solve or C-product per share)
ers_status group_apply(ers_ctx* g, const double* b, double* x, bool solve) {
  std::vector<std::vector<double>> bs, xs(g->group.size());
  split_state(g, b, bs);
  for (size_t q = 0; q < g->group.size(); ++q) xs[q].assign(bs[q].size(), 0.0);
  ers_status st = group_each(g, [&](ers_ctx* s, int q) {
    return solve ? ers_solve(s, bs[q].data(), xs[q].data())
                 : ers_spmv_C(s, bs[q].data(), xs[q].data());
  });
  if (st != ERS_OK) return st;
  join_state(g, xs, x);
  return ERS_OK;
}

ers_status group_get_state_inst(ers_ctx* g, int32_t k, double* t, double* x, double* h) {
  if (k < 0 || k >= g->ninst) return group_fail(g, ERS_ERR_INVALID, "instance index out of range");
  int q = g->inst_grp[k];
  DeviceGuard dg(g->group_dev[q]);
  ers_status st = ers_get_state_inst(g->group[q], g->inst_loc[k], t, x, h);
  if (st != ERS_OK) g->err = g->group[q]->err;
  return st;
}

ers_status group_records(ers_ctx* g, int32_t k, ers_step_record* out, int32_t cap,
                         int32_t* count) {
  if (k < 0 || k >= g->ninst) return group_fail(g, ERS_ERR_INVALID, "instance index out of range");
  return ers_batch_records(g->group[g->inst_grp[k]], g->inst_loc[k], out, cap, count);
}

// training samples in the same order as one batched context of the whole batch: instance by
// instance in input order
ers_status group_samples(ers_ctx* g, float* X, float* T, int32_t cap, int32_t* count) {
  int64_t ns = 0;
  for (int k = 0; k < g->ninst; ++k) {
    const auto& R = g->group[g->inst_grp[k]]->recs[g->inst_loc[k]];
    for (size_t a = 0; a + 1 < R.size(); ++a) {
      float t[2];
      if (!ctrl_target(R.data(), (int)a + 1, R[a + 1], t)) continue;
      if (X && T && ns < cap) {
        ctrl_features(R.data(), (int)a + 1, X + ns * ERS_CTRL_FEATURES);
        T[2 * ns] = t[0];
        T[2 * ns + 1] = t[1];
      }
      ++ns;
    }
  }
  if (count) *count = (int32_t)std::min<int64_t>(ns, INT32_MAX);
  return ERS_OK;
}

// every share gets its own copy of the network on its device (shares run concurrently)
ers_status group_set_controller(ers_ctx* g, ers_mlp* mlp, int32_t parts, double margin) {
  std::vector<float> P;
  if (mlp) {
    P.assign(ers_mlp_nparam(), 0.0f);
    ers_status st = ers_mlp_get_params(mlp, P.data());
    if (st != ERS_OK) return group_fail(g, st, std::string("network: ") + ers_mlp_last_error(mlp));
  }
  g->group_nets.resize(g->group.size(), nullptr);
  return group_each(g, [&](ers_ctx* s, int q) {
    ers_mlp*& net = g->group_nets[q];
    if (mlp && !net) {
      ers_status st = ers_mlp_create(&net, 0);
      if (st != ERS_OK) return ctx_fail(s, st, "network copy: allocation failed");
    }
    if (mlp) {
      ers_status st = ers_mlp_set_params(net, P.data());
      if (st != ERS_OK) return ctx_fail(s, st, "network copy: parameters");
    }
    return ers_batch_set_controller(s, mlp ? net : nullptr, parts, margin);
  });
}

ers_status group_stats(ers_ctx* g, ers_stats_t* out) {
  ers_stats_t acc{};
  ers_status st = group_each(g, [&](ers_ctx* s, int) {
    ers_stats_t x{};
    ers_status r = ers_stats(s, &x);
    if (r != ERS_OK) return r;
    acc.steps = std::max(acc.steps, x.steps);
    acc.rejects += x.rejects;
    acc.refactors += x.refactors;
    acc.krylov_vectors += x.krylov_vectors;
    acc.solves += x.solves;
    acc.n += x.n;
    acc.nsn += x.nsn;
    acc.nlevels = std::max(acc.nlevels, x.nlevels);
    acc.etree_height = std::max(acc.etree_height, x.etree_height);
    acc.max_front = std::max(acc.max_front, x.max_front);
    acc.nnz_L += x.nnz_L;
    acc.factor_doubles += x.factor_doubles;
    acc.arena_doubles += x.arena_doubles;
    acc.refactor_flops += x.refactor_flops;
    acc.kernel_launches += x.kernel_launches;
    acc.solve_passes += x.solve_passes;
    acc.solve_rhs += x.solve_rhs;
    acc.solve_ms += x.solve_ms;
    acc.solve_bytes_per_pass += x.solve_bytes_per_pass;
    acc.solve_fma_per_rhs += x.solve_fma_per_rhs;
    acc.graph_launches += x.graph_launches;
    acc.merged_blocks += x.merged_blocks;
    acc.merged_columns += x.merged_columns;
    acc.merged_inverse_doubles += x.merged_inverse_doubles;
    acc.merged_inverse_flops += x.merged_inverse_flops;
    acc.host_syncs += x.host_syncs;
    acc.host_polls += x.host_polls;
    return ERS_OK;
  });
  if (st == ERS_OK) *out = acc;
  return st;
}

ers_status group_ctrl_stats(ers_ctx* g, int64_t* proposals, int64_t* rejected, int64_t* kv) {
  int64_t p = 0, r = 0, v = 0;
  for (ers_ctx* s : g->group) {
    p += s->ctrl_proposals;
    r += s->ctrl_rejected;
    v += s->stats.krylov_vectors;
  }
  if (proposals) *proposals = p;
  if (rejected) *rejected = r;
  if (kv) *kv = v;
  return ERS_OK;
}

}  // namespace ers

extern "C" ers_status ers_partition_lpt(const double* cost, int32_t n, int32_t nparts,
                                        int32_t* part_of) {
  if (n < 0 || nparts < 1 || (n > 0 && (!cost || !part_of))) return ERS_ERR_INVALID;
  for (int32_t i = 0; i < n; ++i)
    if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return ERS_ERR_INVALID;
  ers::lpt_partition(cost, n, nparts, part_of);
  return ERS_OK;
}
