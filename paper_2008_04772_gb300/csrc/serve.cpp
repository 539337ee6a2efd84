// Request queue with continuous batching: the serving loop around the solver.
//
// Worker threads (one context and stream each) take requests from a FIFO as
// HBM admission allows, so requests that arrive while others run start as soon
// as a slot and memory are free, and their kernels overlap on the device.
// Problems (assembled A, P, Gram) stay resident between requests and are
// evicted least-recently-used when admission needs room; pending requests of
// one problem with equal solver options are merged into one lockstep batch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace cal {
namespace {

constexpr int kMaxBatch = 32;    // lockstep right-hand sides per solve
constexpr int kMaxHeadSkips = 8;  // later requests that may start ahead of a waiting head

// ---- footprint estimate ------------------------------------------------------
struct Footprint {
  int64_t resident = 0;  // spaces, stored A and P blocks, Gram CSR
  int64_t solve = 0;     // per solve of nrhs columns: vectors, Krylov basis, batch state
};

// Device bytes of the blocks the solve assembles (dense A on the union and per
// scatterer; P per scatterer, dense or near-field), following the storage of
// the assembly: complex64 (8 B) or complex128 (16 B) entries, S and C.
int64_t resident_bytes(const Mesh& m, const std::vector<double>& area_m, const cal_solve_opts& o) {
  const int64_t esz = o.precision == CAL_FP64 ? 16 : 8;
  const int64_t N = m.ne;
  int64_t b = 0;
  if (o.matrix_free) {
    // only touching-pair entries, S and C, at k_e and at k_m: about 30 edges
    // reach one edge through touching triangles at valence 6; 40 per row taken
    b += 2 * (2 * N * 40 * esz + N * 40 * 4 + (N + 1) * 8);
  } else {
    b += 2 * N * N * esz;  // S, C at k_e on the union
    for (int64_t d = 0; d < m.M; ++d) {
      const int64_t n = m.edge_off[d + 1] - m.edge_off[d];
      b += 2 * n * n * esz;  // S, C at k_m
    }
    if (o.precision != CAL_FP64) b += 3 * N * N * 8;  // combined float32 blocks of A
  }
  if (o.precond != CAL_PRECOND_NONE) {
    const int pc = o.precond;
    const int sides = pc == CAL_PRECOND_D ? 2 : 1;
    const int ops = (pc == CAL_PRECOND_SE || pc == CAL_PRECOND_SI) ? 1 : 2;
    for (int64_t d = 0; d < m.M; ++d) {
      const int64_t n = m.edge_off[d + 1] - m.edge_off[d];
      int64_t nnz = n * n;
      int64_t idx = 0;
      if (std::isfinite(o.near_cutoff_P)) {
        // pairs whose support boxes are at most chi apart: with supports of
        // about 2h across, count the edges in a disc of radius chi + 2h
        const double chi = o.near_cutoff_P * m.h;
        const double rho = area_m[d] > 0 ? (double)n / area_m[d] : 0.0;
        const double r = chi + 2.0 * m.h;
        const double row = std::min<double>((double)n, rho * M_PI * r * r);
        nnz = std::min<int64_t>(n * n, (int64_t)(row * (double)n));
        idx = (n + 1) * 8 + nnz * 4;
      }
      b += sides * (ops * nnz * esz + idx);
      if (pc == CAL_PRECOND_D && o.precision != CAL_FP64 && !std::isfinite(o.near_cutoff_P))
        b += 3 * n * n * 8;  // combined float32 blocks of P
    }
    b += 2 * ((N + 1) * 8 + 40 * N * 12);  // Gram G and G^T (about 40 entries per row)
    b += m.nt * 6 * 256;                    // barycentric space records
  }
  b += m.nt * 256;  // primal space records
  return b;
}

int64_t solve_bytes(const Mesh& m, const cal_solve_opts& o, int64_t nrhs, int64_t ndir, int64_t resident) {
  const int64_t N = m.ne, n2 = 2 * N, z = 16;
  const int64_t nb = std::min<int64_t>(nrhs, kMaxBatch);
  const int64_t mk = std::max(1, std::min(o.restart, o.maxit));
  int64_t b = 2 * nrhs * n2 * z;                  // right-hand sides and solution
  b += 4 * nb * n2 * z;                           // preconditioned rhs, residual, batch padding
  b += nb * (mk + 1) * n2 * z + 3 * nb * n2 * z;  // Krylov basis and GMRES vectors
  b += nb * (mk + 1) * mk * z;                    // Hessenberg matrices
  b += 4 * nb * n2 * z;                           // work vectors of the batch, interleaved copy for CSR blocks
  if (o.precision != CAL_FP64 && nb >= 4) {
    const int64_t NB = ((4 * nb + 15) / 16) * 16;
    b += 3 * NB * 2 * N * 4 + 2 * N * NB * 4;  // tensor-core operands (and their split) and outputs
    b += 2 * resident;                         // split copies of the dense blocks
  }
  if (o.precond != CAL_PRECOND_NONE) {
    const int64_t c = o.precision == CAL_FP64 ? 16 : 8;
    b += 2 * (40 * N * c / 2 + 10 * 2 * nb * N * c);  // Gram solvers
  }
  b += nrhs * ndir * 3 * z + ndir * 24;  // far field
  return b + (64 << 20);                  // allocation rounding and small buffers
}

std::vector<double> scatterer_areas(const std::vector<double>& v, const std::vector<int32_t>& t,
                                    const std::vector<int32_t>& dom, int64_t M) {
  std::vector<double> a(std::max<int64_t>(M, 1), 0.0);
  const int64_t nt = (int64_t)t.size() / 3;
  for (int64_t i = 0; i < nt; ++i) {
    const double* p0 = &v[3 * t[3 * i]];
    const double* p1 = &v[3 * t[3 * i + 1]];
    const double* p2 = &v[3 * t[3 * i + 2]];
    const double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    const double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
    const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const int d = dom.empty() ? 0 : dom[i];
    if (d >= 0 && d < (int)a.size()) a[d] += 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  }
  return a;
}

// ---- requests and resident problems -----------------------------------------------
struct Request {
  int64_t ticket = 0;
  std::vector<double> verts, eps, mu, inc, dirs;
  std::vector<int32_t> tris, domain;
  double k_ext = 0;
  int64_t nrhs = 0, ndir = 0;
  cal_solve_opts opts{};
  std::string ident;  // every input the assembled operators depend on
  Mesh mesh;          // host mesh (validated at submit)
  Footprint fp;
  cal_request_result res{};
  std::vector<double> far;
  bool done = false;
};

struct Resident {
  std::string ident;
  cal_problem* prob = nullptr;
  int64_t base = 0;   // spaces, blocks and Gram matrices
  int64_t batch = 0;  // batch state the problem keeps between solves
  bool busy = false;
  double last_used = 0;
  int64_t bytes() const { return base + batch; }  // reserved while resident
};

// the solver options that must agree for two requests to share a batch
bool same_solver(const cal_solve_opts& a, const cal_solve_opts& b) {
  return a.tol == b.tol && a.restart == b.restart && a.maxit == b.maxit && a.refine == b.refine &&
         a.rhs_mode == b.rhs_mode;
}

template <typename T>
void append_bytes(std::string& s, const T* p, size_t n) {
  s.append(reinterpret_cast<const char*>(p), n * sizeof(T));
}

}  // namespace
}  // namespace cal

using namespace cal;

struct cal_queue {
  int device = 0;
  int64_t budget = 0;
  std::vector<cal_ctx*> ctxs;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int64_t next_ticket = 1;
  std::deque<Request*> pending;
  std::map<int64_t, std::unique_ptr<Request>> requests;
  std::list<Resident> cache;  // front = most recently used
  std::vector<std::string> creating;  // problems being assembled right now
  int64_t reserved = 0;
  int head_skips = 0;
  int64_t head_ticket = 0;
  cal_queue_stats st{};
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double clock() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  Resident* find(const std::string& ident) {
    for (auto& r : cache)
      if (r.ident == ident) return &r;
    return nullptr;
  }

  // evict idle resident problems (least recently used first) until `need`
  // more bytes fit; never the one in `keep`. Evicts nothing if even evicting
  // every idle problem would not make room.
  bool evict_for(int64_t need, const Resident* keep) {
    int64_t idle = 0;
    for (auto& r : cache)
      if (!r.busy && &r != keep) idle += r.bytes();
    if (reserved - idle + need > budget) return false;
    while (reserved + need > budget) {
      auto victim = cache.end();
      for (auto it = cache.begin(); it != cache.end(); ++it)
        if (!it->busy && &*it != keep && (victim == cache.end() || it->last_used < victim->last_used)) victim = it;
      if (victim == cache.end()) return false;
      cal_problem_destroy(victim->prob);
      reserved -= victim->bytes();
      cache.erase(victim);
      ++st.evictions;
    }
    return true;
  }

  struct Pick {
    std::vector<Request*> group;
    Resident* res = nullptr;  // resident problem to reuse (marked busy)
    int64_t reserve = 0;      // bytes reserved for this run
  };

  // Admission under the lock: the first pending request (FIFO) whose footprint
  // fits; a later one may start ahead of a waiting head only kMaxHeadSkips times.
  bool pick(Pick& p) {
    if (pending.empty()) return false;
    if (pending.front()->ticket != head_ticket) {
      head_ticket = pending.front()->ticket;
      head_skips = 0;
    }
    for (size_t i = 0; i < pending.size(); ++i) {
      if (i > 0 && head_skips >= kMaxHeadSkips) return false;
      Request* r = pending[i];
      Resident* hit = find(r->ident);
      if (hit && hit->busy) continue;  // its operators are in use: wait, then batch
      if (!hit && std::find(creating.begin(), creating.end(), r->ident) != creating.end())
        continue;  // being assembled for another request: wait and reuse it
      // merge pending requests of the same problem and solver options
      std::vector<Request*> group{r};
      int64_t cols = r->nrhs;
      for (size_t j = i + 1; j < pending.size() && cols < kMaxBatch; ++j) {
        Request* o = pending[j];
        if (o->ident == r->ident && same_solver(o->opts, r->opts) && cols + o->nrhs <= kMaxBatch) {
          group.push_back(o);
          cols += o->nrhs;
        }
      }
      int64_t ndir = 0;
      for (Request* g : group) ndir = std::max(ndir, g->ndir);
      const int64_t need = solve_bytes(r->mesh, r->opts, cols, ndir, r->fp.resident) + (hit ? 0 : r->fp.resident);
      if (reserved + need > budget && !evict_for(need, hit)) continue;
      // admitted
      if (i > 0) ++head_skips;
      for (Request* g : group) pending.erase(std::find(pending.begin(), pending.end(), g));
      if (hit) hit->busy = true;
      else creating.push_back(r->ident);
      reserved += need;
      st.peak_reserved_bytes = std::max(st.peak_reserved_bytes, reserved);
      p.group = std::move(group);
      p.res = hit;
      p.reserve = need;
      return true;
    }
    return false;
  }

  void run(cal_ctx* ctx, Pick& p);
  void worker(int slot);
};

void cal_queue::worker(int slot) {
  cal_ctx* ctx = ctxs[slot];
  cudaSetDevice(device);
  for (;;) {
    Pick p;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) return;
        if (pick(p)) break;
        cv_work.wait(lk);
      }
      st.running++;
      st.peak_running = std::max(st.peak_running, st.running);
    }
    run(ctx, p);
    {
      std::lock_guard<std::mutex> lk(mu);
      st.running--;
    }
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

void cal_queue::run(cal_ctx* ctx, Pick& p) {
  Request* r0 = p.group.front();
  const double t_start = clock();
  int rc = CAL_OK;
  cal_problem* prob = p.res ? p.res->prob : nullptr;
  bool reused = prob != nullptr;
  int64_t resident_real = 0;
  if (!prob) {
    // the request's own mesh object (its arrays were copied at submit)
    cal_mesh* mesh = nullptr;
    rc = cal_mesh_create(ctx, r0->verts.data(), (int64_t)r0->verts.size() / 3, r0->tris.data(),
                         (int64_t)r0->tris.size() / 3, r0->domain.empty() ? nullptr : r0->domain.data(), &mesh);
    if (!rc)
      rc = cal_problem_create(ctx, mesh, r0->k_ext, r0->eps.data(), r0->mu.empty() ? nullptr : r0->mu.data(),
                              &r0->opts, &prob);
    cal_mesh_destroy(mesh);
    if (!rc) {
      cal_problem_info pi{};
      cal_problem_get_info(prob, &pi);
      resident_real = pi.bytes_A + pi.bytes_P + pi.bytes_G + r0->mesh.nt * 7 * 256;
    }
  }
  std::vector<double> inc;
  int64_t cols = 0;
  for (Request* g : p.group) {
    inc.insert(inc.end(), g->inc.begin(), g->inc.end());
    cols += g->nrhs;
  }
  cal_solution* sol = nullptr;
  cal_solve_info info{};
  if (!rc) {
    rc = cal_problem_solve(ctx, prob, inc.data(), cols, &r0->opts, &sol);
    if (sol) cal_solution_get_info(sol, &info);
  }
  // far field per request, from its own columns
  std::vector<std::vector<double>> far(p.group.size());
  if (sol) {
    int64_t off = 0;
    for (size_t k = 0; k < p.group.size(); ++k) {
      Request* g = p.group[k];
      std::vector<double> all((size_t)cols * g->ndir * 6);
      const int frc = cal_farfield(sol, g->dirs.data(), g->ndir, all.data());
      if (frc) {
        if (!rc || rc == CAL_ENOTCONV) rc = frc;
      } else {
        far[k].assign(all.begin() + off * g->ndir * 6, all.begin() + (off + g->nrhs) * g->ndir * 6);
      }
      off += g->nrhs;
    }
    cal_solution_destroy(sol);
  }
  int64_t batch_bytes = 0;
  if (prob) {
    cal_problem_info pi{};
    cal_problem_get_info(prob, &pi);
    batch_bytes = pi.bytes_batch;
  }
  const double t_done = clock();
  std::lock_guard<std::mutex> lk(mu);
  // reservations: the solve's temporaries (and a new problem's estimate) go;
  // a problem that solved stays resident at its real size plus its batch state
  reserved -= p.reserve;
  if (!p.res) creating.erase(std::find(creating.begin(), creating.end(), r0->ident));
  const bool ok = prob && (rc == CAL_OK || rc == CAL_ENOTCONV);
  if (p.res) {
    reserved -= p.res->bytes();
    if (ok) {
      p.res->batch = batch_bytes;
      p.res->busy = false;
      p.res->last_used = t_done;
      reserved += p.res->bytes();
    } else {
      for (auto it = cache.begin(); it != cache.end(); ++it)
        if (&*it == p.res) {
          cache.erase(it);
          break;
        }
      cal_problem_destroy(prob);
    }
  } else if (ok) {
    cache.push_front(Resident{});
    Resident& e = cache.front();
    e.ident = r0->ident;
    e.prob = prob;
    e.base = resident_real;
    e.batch = batch_bytes;
    e.last_used = t_done;
    reserved += e.bytes();
    ++st.problems_created;
  } else if (prob) {
    cal_problem_destroy(prob);
  }
  st.peak_reserved_bytes = std::max(st.peak_reserved_bytes, reserved);
  ++st.batches;
  if (reused) st.problem_hits += (int64_t)p.group.size();
  st.merged += (int64_t)p.group.size() - 1;
  for (size_t k = 0; k < p.group.size(); ++k) {
    Request* g = p.group[k];
    g->res.status = rc;
    g->res.iterations = info.iterations;
    g->res.residual = info.residual;
    g->res.t_start = t_start;
    g->res.t_done = t_done;
    g->res.footprint_bytes = p.reserve;
    g->res.batch_rhs = (int32_t)cols;
    g->res.reused = reused ? 1 : 0;
    g->far = std::move(far[k]);
    g->done = true;
    ++st.completed;
  }
}

extern "C" {

int cal_request_footprint(const cal_request* req, int64_t* resident, int64_t* solve) {
  if (!req || !req->verts || !req->tris || req->nv < 3 || req->nt < 1 || req->nrhs < 1)
    return fail(CAL_EINVAL, "cal_request_footprint: bad request");
  Mesh m;
  int rc = build_mesh(m, req->verts, req->nv, req->tris, req->nt, req->domain);
  if (rc) return rc;
  std::vector<double> v(req->verts, req->verts + 3 * req->nv);
  std::vector<int32_t> t(req->tris, req->tris + 3 * req->nt), d;
  if (req->domain) d.assign(req->domain, req->domain + req->nt);
  const std::vector<double> area = scatterer_areas(v, t, d, m.M);
  if (resident) *resident = resident_bytes(m, area, req->opts);
  const int64_t res = resident_bytes(m, area, req->opts);
  if (solve) *solve = solve_bytes(m, req->opts, req->nrhs, std::max<int64_t>(req->ndir, 0), res);
  return CAL_OK;
}

int cal_queue_create(int device, size_t hbm_budget_bytes, int slots, cal_queue** out) {
  if (!out || slots < 1 || slots > 64) return fail(CAL_EINVAL, "cal_queue_create: need out and 1 <= slots <= 64");
  auto q = std::make_unique<cal_queue>();
  q->device = device;
  int rc = CAL_OK;
  cal_ctx* first = nullptr;  // also checks the device
  if ((rc = cal_init(&first, device))) return rc;
  q->ctxs.push_back(first);
  if (hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cal_ctx_destroy(first);
      return fail(CAL_ECUDA, "cal_queue_create: cudaMemGetInfo failed");
    }
    hbm_budget_bytes = (size_t)(0.85 * (double)fr);
  }
  q->budget = (int64_t)hbm_budget_bytes;
  q->st.budget_bytes = q->budget;
  q->st.slots = slots;
  for (int s = 1; s < slots; ++s) {
    cal_ctx* c = nullptr;
    if ((rc = cal_init(&c, device))) {
      for (cal_ctx* x : q->ctxs) cal_ctx_destroy(x);
      return rc;
    }
    q->ctxs.push_back(c);
  }
  cal_queue* qp = q.release();
  for (int s = 0; s < slots; ++s) qp->workers.emplace_back([qp, s] { qp->worker(s); });
  *out = qp;
  return CAL_OK;
}

int cal_queue_submit(cal_queue* q, const cal_request* req, int64_t* ticket) {
  if (!q || !req || !ticket) return fail(CAL_EINVAL, "cal_queue_submit: NULL argument");
  if (!req->verts || !req->tris || !req->eps_r || !req->inc || !req->dirs || req->nrhs < 1 || req->ndir < 1 ||
      req->nv < 3 || req->nt < 1)
    return fail(CAL_EINVAL, "cal_queue_submit: incomplete request");
  auto r = std::make_unique<Request>();
  int rc = build_mesh(r->mesh, req->verts, req->nv, req->tris, req->nt, req->domain);
  if (rc) return rc;
  const int64_t M = r->mesh.M;
  r->verts.assign(req->verts, req->verts + 3 * req->nv);
  r->tris.assign(req->tris, req->tris + 3 * req->nt);
  if (req->domain) r->domain.assign(req->domain, req->domain + req->nt);
  r->k_ext = req->k_ext;
  r->eps.assign(req->eps_r, req->eps_r + 2 * M);
  if (req->mu_r) r->mu.assign(req->mu_r, req->mu_r + 2 * M);
  r->inc.assign(req->inc, req->inc + 6 * req->nrhs);
  r->dirs.assign(req->dirs, req->dirs + 3 * req->ndir);
  r->nrhs = req->nrhs;
  r->ndir = req->ndir;
  r->opts = req->opts;
  // identity of the assembled operators: mesh, wavenumber, materials and the
  // options that change assembly
  std::string& id = r->ident;
  append_bytes(id, r->verts.data(), r->verts.size());
  append_bytes(id, r->tris.data(), r->tris.size());
  append_bytes(id, r->domain.data(), r->domain.size());
  append_bytes(id, &r->k_ext, 1);
  append_bytes(id, r->eps.data(), r->eps.size());
  append_bytes(id, r->mu.data(), r->mu.size());
  const cal_solve_opts& o = r->opts;
  const int32_t ai[8] = {o.precond,     o.precision,   o.q_regular_A, o.q_singular_A,
                         o.q_regular_P, o.q_singular_P, o.matrix_free, o.discretisation};
  append_bytes(id, ai, 8);
  append_bytes(id, &o.near_cutoff_P, 1);
  append_bytes(id, &o.aca_nu_P, 1);
  const std::vector<double> area = scatterer_areas(r->verts, r->tris, r->domain, M);
  r->fp.resident = resident_bytes(r->mesh, area, o);
  r->fp.solve = solve_bytes(r->mesh, o, r->nrhs, r->ndir, r->fp.resident);
  if (r->fp.resident + r->fp.solve > q->budget)
    return fail(CAL_ENOMEM, "cal_queue_submit: request needs ~%lld bytes, above the budget of %lld",
                (long long)(r->fp.resident + r->fp.solve), (long long)q->budget);
  {
    std::lock_guard<std::mutex> lk(q->mu);
    r->ticket = q->next_ticket++;
    r->res.t_submit = q->clock();
    *ticket = r->ticket;
    q->pending.push_back(r.get());
    q->requests[r->ticket] = std::move(r);
    ++q->st.submitted;
  }
  q->cv_work.notify_all();
  return CAL_OK;
}

int cal_queue_wait(cal_queue* q, int64_t ticket, double timeout_s, cal_request_result* res, double* farfield) {
  if (!q) return fail(CAL_EINVAL, "cal_queue_wait: NULL queue");
  std::unique_lock<std::mutex> lk(q->mu);
  auto it = q->requests.find(ticket);
  if (it == q->requests.end()) return fail(CAL_EINVAL, "cal_queue_wait: unknown ticket %lld", (long long)ticket);
  Request* r = it->second.get();
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) {
    q->cv_done.wait(lk, ready);
  } else if (!q->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return fail(CAL_ETIMEOUT, "cal_queue_wait: request %lld not finished after %.3f s", (long long)ticket, timeout_s);
  }
  if (res) *res = r->res;
  if (farfield && !r->far.empty()) std::memcpy(farfield, r->far.data(), r->far.size() * sizeof(double));
  q->requests.erase(it);
  return CAL_OK;
}

int cal_queue_poll(cal_queue* q, int64_t ticket, int* state) {
  if (!q || !state) return fail(CAL_EINVAL, "cal_queue_poll: NULL argument");
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->requests.find(ticket);
  if (it == q->requests.end()) return fail(CAL_EINVAL, "cal_queue_poll: unknown ticket %lld", (long long)ticket);
  const Request* r = it->second.get();
  if (r->done) *state = CAL_REQ_DONE;
  else if (std::find(q->pending.begin(), q->pending.end(), r) != q->pending.end()) *state = CAL_REQ_PENDING;
  else *state = CAL_REQ_RUNNING;
  return CAL_OK;
}

int cal_queue_get_stats(cal_queue* q, cal_queue_stats* stats) {
  if (!q || !stats) return fail(CAL_EINVAL, "cal_queue_get_stats: NULL argument");
  std::lock_guard<std::mutex> lk(q->mu);
  *stats = q->st;
  stats->reserved_bytes = q->reserved;
  stats->pending = (int32_t)q->pending.size();
  return CAL_OK;
}

void cal_queue_destroy(cal_queue* q) {
  if (!q) return;
  {
    std::lock_guard<std::mutex> lk(q->mu);
    q->stop = true;
    q->pending.clear();
  }
  q->cv_work.notify_all();
  for (auto& w : q->workers) w.join();
  for (auto& e : q->cache) cal_problem_destroy(e.prob);
  q->cache.clear();
  for (cal_ctx* c : q->ctxs) cal_ctx_destroy(c);
  delete q;
}

}  // extern "C"
