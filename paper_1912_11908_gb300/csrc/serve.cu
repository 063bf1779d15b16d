// Continuous-batching request loop over many cases on one GPU (C ABI in
// include/ibm.h: ibm_server_*).
//
// Requests (body, grid, flow, motion, number of steps) wait in a host queue
// and are admitted while a slot and enough device memory are free; each
// admitted case owns its device state, tags and lists.
//
// Batched mode (default) for FP32-bulk cases: the requests admitted in one
// pass of the loop form groups of cases of similar size (grids within a factor
// four in cells), equal step counts, the same time scheme (explicit RK3, or
// dual time with equal sub-iteration counts) and the same stage-kernel variant
// (WENO5 or TVD-2, linear or quadratic reconstruction; dual-time groups the
// first of each), up to MAX_BATCH cases per group.
// One step of a group is one CUDA graph: the per-case work that precedes the
// stages (re-classification and stencils of moving bodies, the force and
// acceleration of a body under the fluid force, dt, or the rotation of a
// dual-time case's time levels) forked onto the cases' own streams, then per
// RK stage (per pseudo stage of every sub-iteration) ONE launch over the block
// table of all member cases, then the per-case work that ends the step (the
// body update of Eq. 10, the end of a dual-time step), forked likewise.  A group's membership is fixed when it forms, so its graph is
// captured once and its members finish together; requests that arrive later
// form new groups, which run beside the old ones on their own streams.  A small
// autotuner picks the plain-tile launch's schedule (one block per table entry,
// or a persistent grid striding over the table) by timing the candidates on
// the group itself, once per size class and membership size.
//
// Other cases (FP64; dual time with TVD-2 or the quadratic reconstruction),
// and every case when batching is off, advance on their own streams in chunks
// of steps replayed from their own graphs.
//
// A case that has taken all its steps is retired: its forces and time are
// read, its memory freed, and the next waiting request can take the slot.
// Cases share nothing on the device and every kernel is deterministic, so a
// request gives the same result alone and in any mix: bit for bit on its own
// stream (the kernels of a case stepped alone), and up to FP32 rounding in a
// group, whose block-table kernels compile the same per-tile source
// separately (fused multiply-adds may round differently).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "ibm_internal.cuh"

extern "C" ibm_status ibm__noalloc_fail(ibm_status s, const char *msg);  // sets ibm_last_error()

namespace {

using namespace ibm;

struct Request {
  int64_t id;
  std::vector<double> verts;
  ibm_geometry geo;
  ibm_grid grid;
  ibm_flow flow;
  ibm_motion motion;
  int nsteps;
  size_t bytes;
  ibm_result res;
};

struct Group;

struct Active {
  Request *req = nullptr;
  ibm_case *c = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;  // own-stream mode: recorded after the last enqueued chunk
  cudaEvent_t join = nullptr;  // batched mode: end of the case's pre-stage work inside the group step
  int launched = 0;            // steps enqueued so far
  Group *group = nullptr;
  bool prestage = false;       // has per-step work before the stages
  bool poststage = false;      // has per-step work after the stages
};

struct Group {
  int bucket = 0;
  int subiters = 0;  // dual-time sub-iterations per physical step (0: explicit RK3)
  bool coupled = false;  // a member's body moves under the fluid force
  std::vector<Active *> members;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool dirty = true;
  long long graph_kernels = 0;
  int plain_grid = 0;
  StageBatch *batch = nullptr;  // the group's block table (kernel parameter of the stage launches)
};

double now_s(const std::chrono::steady_clock::time_point &t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// size class: cell counts within a factor four share a group
int bucket_of(const Request *r) {
  const double cells = (double)r->grid.nx * (double)r->grid.ny;
  return (int)std::floor(std::log2(cells) / 2.0);
}

}  // namespace

struct ibm_server {
  size_t budget = 0, used = 0;
  int max_active = 0;
  int chunk = 0;
  int mode = IBM_SERVE_BATCHED | IBM_SERVE_AUTOTUNE;
  int64_t next_id = 1;
  int nsms = 152;
  std::chrono::steady_clock::time_point t0;
  std::deque<Request *> pending;
  std::vector<Active *> active;
  std::vector<Group *> groups;
  std::map<int64_t, Request *> all;
  std::map<int, int> tuned;  // (size class, membership class) -> plain-tile grid (0: one block per entry)
  int64_t stats[IBM_SERVER_NSTATS] = {};
};

static void group_destroy(Group *g) {
  if (g->graph) cudaGraphExecDestroy(g->graph);
  for (cudaEvent_t e : {g->fork, g->done, g->t0, g->t1})
    if (e) cudaEventDestroy(e);
  if (g->s) cudaStreamDestroy(g->s);
  delete g->batch;
  delete g;
}

static Group *group_create(int bucket) {
  Group *g = new (std::nothrow) Group();
  if (!g) return nullptr;
  g->bucket = bucket;
  g->batch = new (std::nothrow) StageBatch();
  cudaError_t e = g->batch ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking);
  for (cudaEvent_t *ev : {&g->fork, &g->done})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&g->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&g->t1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    group_destroy(g);
    return nullptr;
  }
  return g;
}

extern "C" ibm_status ibm_server_create(size_t device_bytes_budget, int max_active, int steps_per_chunk,
                                        ibm_server **out) {
  if (!out || max_active < 1 || steps_per_chunk < 1)
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_create: bad arguments");
  ibm_server *s = new (std::nothrow) ibm_server();
  if (!s) return ibm__noalloc_fail(IBM_ENOMEM, "ibm_server_create: host allocation failed");
  if (device_bytes_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      cudaGetLastError();
      return ibm__noalloc_fail(IBM_ECUDA, "ibm_server_create: cudaMemGetInfo failed");
    }
    device_bytes_budget = fr / 10 * 8;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s->nsms, cudaDevAttrMultiProcessorCount, dev);
  s->budget = device_bytes_budget;
  s->max_active = max_active;
  s->chunk = steps_per_chunk;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return IBM_OK;
}

extern "C" ibm_status ibm_server_set_mode(ibm_server *s, int mode) {
  if (!s || (mode & ~(IBM_SERVE_BATCHED | IBM_SERVE_AUTOTUNE)))
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_set_mode: bad arguments");
  if (!s->all.empty()) return ibm__noalloc_fail(IBM_ESTATE, "ibm_server_set_mode: requests already submitted");
  s->mode = mode;
  return IBM_OK;
}

extern "C" ibm_status ibm_server_stats(const ibm_server *s, int64_t *out, int n) {
  if (!s || !out || n < 0 || n > IBM_SERVER_NSTATS) return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_stats: bad arguments");
  for (int q = 0; q < n; q++) out[q] = s->stats[q];
  return IBM_OK;
}

extern "C" ibm_status ibm_server_submit(ibm_server *s, const ibm_geometry *geo, const ibm_grid *grid,
                                        const ibm_flow *flow, const ibm_motion *motion, int nsteps, int64_t *id) {
  if (!s || !geo || !grid || !flow || !id || nsteps < 0)
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_submit: bad arguments");
  size_t bytes = ibm_case_device_bytes(geo, grid, flow, motion);
  if (bytes == 0) return IBM_EINVAL;  // ibm_case_device_bytes validated and set the message
  if (bytes > s->budget) return ibm__noalloc_fail(IBM_ENOMEM, "ibm_server_submit: request exceeds the memory budget");
  Request *r = new (std::nothrow) Request();
  if (!r) return ibm__noalloc_fail(IBM_ENOMEM, "ibm_server_submit: host allocation failed");
  r->id = s->next_id++;
  r->verts.assign(geo->verts, geo->verts + 2 * (size_t)(geo->nverts > 0 ? geo->nverts : 0));
  r->geo = *geo;
  r->geo.verts = r->verts.empty() ? nullptr : r->verts.data();
  r->grid = *grid;
  r->flow = *flow;
  if (motion) r->motion = *motion;
  else std::memset(&r->motion, 0, sizeof r->motion);
  r->nsteps = nsteps;
  r->bytes = bytes;
  std::memset(&r->res, 0, sizeof r->res);
  r->res.id = r->id;
  r->res.state = IBM_REQ_PENDING;
  r->res.submit_s = now_s(s->t0);
  s->pending.push_back(r);
  s->all[r->id] = r;
  *id = r->id;
  return IBM_OK;
}

// Read the result, free the case and drop it from its group (the group graph
// is re-captured before its next launch).  The case's work must be complete.
static void retire(ibm_server *s, Active *a, ibm_status st) {
  Request *r = a->req;
  if (st == IBM_OK) st = ibm_forces(a->c, r->res.forces);
  double tt[2] = {0.0, 0.0};
  if (st == IBM_OK) st = ibm_get_state(a->c, IBM_TIME, tt, sizeof tt, 0);
  r->res.t = tt[0];
  r->res.steps_done = a->launched;
  r->res.status = st;
  r->res.state = st == IBM_OK ? IBM_REQ_DONE : IBM_REQ_FAILED;
  r->res.finish_s = now_s(s->t0);
  if (a->group) {
    auto &m = a->group->members;
    m.erase(std::remove(m.begin(), m.end(), a), m.end());
    a->group->dirty = true;
  }
  ibm_destroy_case(a->c);
  if (a->done) cudaEventDestroy(a->done);
  if (a->join) cudaEventDestroy(a->join);
  cudaStreamDestroy(a->stream);
  s->used -= r->bytes;
  s->active.erase(std::remove(s->active.begin(), s->active.end(), a), s->active.end());
  delete a;
}

// the group's table: member descriptors and tile offsets (kernel parameters of the stage launches)
static void build_table(Group *g) {
  const int n = (int)g->members.size();
  StageCase cs[MAX_BATCH];
  for (int q = 0; q < n; q++) case_stage_desc(g->members[q]->c, &cs[q]);
  build_stage_batch(cs, n, g->batch);
}

// Capture one step of the group: pre-stage work of each member on its own
// stream, then the three batched stages (one launch each over the combined table).
static ibm_status capture_group(ibm_server *s, Group *g) {
  build_table(g);
  const StageBatch &b = *g->batch;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(g->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return ibm__noalloc_fail(IBM_ECUDA, "request loop: stream capture failed");
  }
  long long nk = 0;
  bool any_pre = false;
  for (Active *a : g->members) any_pre |= a->prestage;
  if (any_pre) {
    cudaEventRecord(g->fork, g->s);
    for (Active *a : g->members) {
      if (!a->prestage) continue;
      cudaStreamWaitEvent(a->stream, g->fork, 0);
      nk += case_enqueue_prestage(a->c);
      cudaEventRecord(a->join, a->stream);
      cudaStreamWaitEvent(g->s, a->join, 0);
    }
  }
  // one launch per stage over the combined table, stages chained by programmatic launch
  const bool nonempty = b.plain_start[b.n] + b.body_start[b.n] > 0;
  if (g->subiters > 0) {
    for (int it = 0; it < g->subiters; it++)
      for (int st = 1; st <= 3; st++) {
        launch_dual_f32_batch_one(b, st, g->plain_grid, true, g->s);
        nk += nonempty;
      }
  } else {
    for (int st = 1; st <= 3; st++) {
      launch_stage_f32_batch_one(b, st, g->plain_grid, true, g->s);
      nk += nonempty;
    }
  }
  bool any_post = false;
  for (Active *a : g->members) any_post |= a->poststage;
  if (any_post) {
    cudaEventRecord(g->fork, g->s);
    for (Active *a : g->members) {
      if (!a->poststage) continue;
      cudaStreamWaitEvent(a->stream, g->fork, 0);
      nk += case_enqueue_poststage(a->c);
      cudaEventRecord(a->join, a->stream);
      cudaStreamWaitEvent(g->s, a->join, 0);
    }
  }
  cudaError_t e = cudaStreamEndCapture(g->s, &graph);
  if (e == cudaSuccess && g->graph) {
    // same topology (only the table and pointers changed): update the executable graph in place
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(g->graph, graph, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(g->graph);
      g->graph = nullptr;
    }
  }
  if (e == cudaSuccess && !g->graph) e = cudaGraphInstantiate(&g->graph, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->graph = nullptr;
    cudaGetLastError();
    return ibm__noalloc_fail(IBM_ECUDA, "request loop: group graph capture failed");
  }
  g->graph_kernels = nk;
  g->dirty = false;
  s->stats[0]++;
  return IBM_OK;
}

// Autotuner: time stage 1 over the group's combined table under each
// candidate schedule and keep the fastest for this size class and membership
// size.  Between steps stage 1 is free of side effects on the solution: it
// reads the mirror of U^n and writes the stage-1 array, the stage times and
// U^n on IB / ghost nodes, all of which the next step's stage 1 rewrites with
// the same values.  Groups whose step reads those IB / ghost values before
// stage 1 rewrites them (the force of a body under the fluid force) and
// dual-time groups (a pseudo stage updates the FP64 iterates) keep one block
// per table entry and are not timed.
static void autotune(ibm_server *s, Group *g) {
  if (g->subiters > 0 || g->coupled) {
    g->plain_grid = 0;
    return;
  }
  int mclass = 0;
  while ((2 << mclass) <= (int)g->members.size()) mclass++;
  const int key = g->bucket * 16 + mclass;
  auto it = s->tuned.find(key);
  if (it != s->tuned.end()) {
    g->plain_grid = it->second;
    return;
  }
  const int entries = g->batch->plain_start[g->batch->n] + g->batch->body_start[g->batch->n];
  const int cands[3] = {0, 6 * s->nsms, 3 * s->nsms};
  int best = 0;
  float best_ms = 1e30f;
  for (int ci = 0; ci < 3; ci++) {
    const int grid = cands[ci];
    if (ci > 0 && grid >= entries) continue;
    launch_stage_f32_batch_one(*g->batch, 1, grid, true, g->s);  // warm-up
    cudaEventRecord(g->t0, g->s);
    for (int rep = 0; rep < 3; rep++) launch_stage_f32_batch_one(*g->batch, 1, grid, true, g->s);
    cudaEventRecord(g->t1, g->s);
    cudaEventSynchronize(g->t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->t0, g->t1);
    if (ms < best_ms) {
      best_ms = ms;
      best = grid;
    }
  }
  cudaGetLastError();
  s->tuned[key] = best;
  g->plain_grid = best;
  s->stats[3]++;
}

extern "C" ibm_status ibm_server_progress(ibm_server *s, int *n_active, int *n_pending) {
  if (!s) return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_progress: server is NULL");
  // 1. retire: own-stream cases whose last chunk finished, group members whose group step finished
  std::vector<Active *> snapshot = s->active;
  for (Active *a : snapshot) {
    cudaError_t q = a->group ? cudaEventQuery(a->group->done) : cudaEventQuery(a->done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) {
      cudaGetLastError();
      retire(s, a, IBM_ECUDA);
    } else if (a->launched >= a->req->nsteps) {
      retire(s, a, a->req->res.status == IBM_OK ? IBM_OK : (ibm_status)a->req->res.status);
    }
  }
  for (size_t k = 0; k < s->groups.size();) {
    if (s->groups[k]->members.empty() && cudaEventQuery(s->groups[k]->done) != cudaErrorNotReady) {
      cudaGetLastError();
      group_destroy(s->groups[k]);
      s->groups.erase(s->groups.begin() + (long)k);
    } else {
      k++;
    }
  }
  // 2. admit waiting requests, in arrival order, while a slot and memory are free.  Batchable requests
  // admitted in this pass form new groups by (size class, steps): a group's membership is fixed when it
  // is formed, so its step graph is captured once and all its members finish together.
  std::map<std::tuple<int, int, int, int>, Group *> forming;
  while (!s->pending.empty() && (int)s->active.size() < s->max_active &&
         s->used + s->pending.front()->bytes <= s->budget) {
    Request *r = s->pending.front();
    s->pending.pop_front();
    Active *a = new (std::nothrow) Active();
    ibm_status st = a ? IBM_OK : IBM_ENOMEM;
    cudaError_t e = cudaSuccess;
    if (st == IBM_OK) e = cudaStreamCreateWithFlags(&a->stream, cudaStreamNonBlocking);
    if (st == IBM_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&a->done, cudaEventDisableTiming);
    if (st == IBM_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&a->join, cudaEventDisableTiming);
    if (st == IBM_OK && e != cudaSuccess) st = IBM_ECUDA;
    if (st == IBM_OK) st = ibm_create_case(&r->geo, &r->grid, &r->flow, &r->motion, a->stream, &a->c);
    const bool batched = st == IBM_OK && (s->mode & IBM_SERVE_BATCHED) && case_batchable(a->c) && r->nsteps > 0;
    if (st == IBM_OK) st = batched ? case_prepare_batch(a->c) : ibm_classify(a->c);
    Group *g = nullptr;
    if (st == IBM_OK && batched) {
      const auto key = std::make_tuple(bucket_of(r), case_subiters(a->c), case_variant(a->c), r->nsteps);
      auto it = forming.find(key);
      if (it != forming.end() && (int)it->second->members.size() < MAX_BATCH) g = it->second;
      if (!g) {
        g = group_create(bucket_of(r));
        if (g) {
          g->subiters = case_subiters(a->c);
          s->groups.push_back(g);
          forming[key] = g;
        } else {
          st = IBM_ECUDA;
        }
      }
    }
    if (st != IBM_OK) {
      cudaGetLastError();
      if (a) {
        if (a->c) ibm_destroy_case(a->c);
        if (a->done) cudaEventDestroy(a->done);
        if (a->join) cudaEventDestroy(a->join);
        if (a->stream) cudaStreamDestroy(a->stream);
        delete a;
      }
      r->res.status = st;
      r->res.state = IBM_REQ_FAILED;
      r->res.finish_s = now_s(s->t0);
      continue;
    }
    r->res.state = IBM_REQ_RUNNING;
    r->res.start_s = now_s(s->t0);
    s->used += r->bytes;
    a->req = r;
    cudaEventRecord(a->done, a->stream);
    if (g) {
      // the group's next step starts after the case's set-up work
      a->group = g;
      // a moving body is re-classified and its dt reduced before the stages of every step (a body under the
      // fluid force also takes the force first and is moved after them); a static body's dt comes from
      // stage 3 (or is fixed); a dual-time step rotates the time levels first and advances t after them
      a->prestage = r->motion.kind != IBM_MOTION_STATIC || g->subiters > 0;
      a->poststage = case_coupled(a->c) || g->subiters > 0;
      g->coupled |= case_coupled(a->c);
      g->members.push_back(a);
      g->dirty = true;
      cudaStreamWaitEvent(g->s, a->done, 0);
    }
    s->active.push_back(a);
  }
  // 3a. own-stream cases: enqueue the next chunk of every case whose previous chunk is done
  for (Active *a : s->active) {
    if (a->group || a->launched >= a->req->nsteps) continue;
    if (cudaEventQuery(a->done) == cudaErrorNotReady) continue;
    const int n = std::min(a->req->nsteps - a->launched, s->chunk);
    ibm_status st = ibm_step(a->c, n);
    if (st != IBM_OK) {
      a->launched = a->req->nsteps;  // retired (as failed) on the next pass
      a->req->res.status = st;
    } else {
      a->launched += n;
    }
    cudaEventRecord(a->done, a->stream);
  }
  // 3b. groups: next chunk of group steps (no member takes more steps than it asked for)
  for (Group *g : s->groups) {
    if (g->members.empty()) continue;
    if (cudaEventQuery(g->done) == cudaErrorNotReady) continue;
    int n = s->chunk;
    for (Active *a : g->members) n = std::min(n, a->req->nsteps - a->launched);
    if (n <= 0) continue;  // a member is finished; it is retired on the next pass
    ibm_status st = IBM_OK;
    if (g->dirty) {
      const auto h0 = std::chrono::steady_clock::now();
      if (s->mode & IBM_SERVE_AUTOTUNE) {
        build_table(g);
        autotune(s, g);
      }
      st = capture_group(s, g);
      s->stats[4] += (int64_t)(1e6 * std::chrono::duration<double>(std::chrono::steady_clock::now() - h0).count());
    }
    for (int q = 0; q < n && st == IBM_OK; q++)
      if (cudaGraphLaunch(g->graph, g->s) != cudaSuccess) st = IBM_ECUDA;
    if (st != IBM_OK) {
      cudaGetLastError();
      for (Active *a : g->members) {
        a->launched = a->req->nsteps;
        a->req->res.status = st;
      }
    } else {
      for (Active *a : g->members) a->launched += n;
      s->stats[1] += n;
      s->stats[2] += n * g->graph_kernels;
    }
    cudaEventRecord(g->done, g->s);
  }
  if (n_active) *n_active = (int)s->active.size();
  if (n_pending) *n_pending = (int)s->pending.size();
  return IBM_OK;
}

extern "C" ibm_status ibm_server_poll(ibm_server *s, int64_t id, ibm_result *out) {
  if (!s || !out) return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_poll: bad arguments");
  auto it = s->all.find(id);
  if (it == s->all.end()) return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_poll: unknown request");
  *out = it->second->res;
  return IBM_OK;
}

extern "C" ibm_status ibm_server_destroy(ibm_server *s) {
  if (!s) return IBM_OK;
  for (Group *g : s->groups) cudaStreamSynchronize(g->s);
  while (!s->active.empty()) {
    Active *a = s->active.back();
    cudaStreamSynchronize(a->stream);
    retire(s, a, IBM_ESTATE);
  }
  for (Group *g : s->groups) group_destroy(g);
  for (auto &kv : s->all) delete kv.second;
  delete s;
  return IBM_OK;
}
