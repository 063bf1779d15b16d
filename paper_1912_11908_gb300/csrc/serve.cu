// Continuous-batching request loop over many cases on one GPU (C ABI in
// include/ibm.h: ibm_server_*).
//
// Requests (body, grid, flow, motion, number of steps) wait in a host queue
// and are admitted while a slot and enough device memory are free; each
// admitted case owns its device state and a stream, is classified once and
// then advanced in chunks of steps (CUDA-graph replays), so the kernels of all
// admitted cases overlap on the device.  A case that has taken all its steps
// is retired: its forces are read, its memory freed, and the next waiting
// request can take the slot.  Requests are independent, so a case gives the
// same result alone and in a mix.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "ibm.h"

extern "C" ibm_status ibm__noalloc_fail(ibm_status s, const char *msg);  // sets ibm_last_error()

namespace {

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

struct Active {
  Request *req;
  ibm_case *c;
  cudaStream_t stream;
  cudaEvent_t done;     // recorded after the last enqueued chunk
  int launched;         // steps enqueued so far
};

double now_s(const std::chrono::steady_clock::time_point &t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct ibm_server {
  size_t budget = 0, used = 0;
  int max_active = 0;
  int chunk = 0;
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  std::deque<Request *> pending;
  std::vector<Active> active;
  std::map<int64_t, Request *> all;
};

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
  s->budget = device_bytes_budget;
  s->max_active = max_active;
  s->chunk = steps_per_chunk;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
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

static void retire(ibm_server *s, size_t k, ibm_status st) {
  Active &a = s->active[k];
  Request *r = a.req;
  if (st == IBM_OK) st = ibm_forces(a.c, r->res.forces);
  double tt[2] = {0.0, 0.0};
  if (st == IBM_OK) st = ibm_get_state(a.c, IBM_TIME, tt, sizeof tt, 0);
  r->res.t = tt[0];
  r->res.steps_done = a.launched;
  r->res.status = st;
  r->res.state = st == IBM_OK ? IBM_REQ_DONE : IBM_REQ_FAILED;
  r->res.finish_s = now_s(s->t0);
  ibm_destroy_case(a.c);
  cudaEventDestroy(a.done);
  cudaStreamDestroy(a.stream);
  s->used -= r->bytes;
  s->active.erase(s->active.begin() + (long)k);
}

extern "C" ibm_status ibm_server_progress(ibm_server *s, int *n_active, int *n_pending) {
  if (!s) return ibm__noalloc_fail(IBM_EINVAL, "ibm_server_progress: server is NULL");
  // retire cases whose last chunk has finished and that have taken all their steps
  for (size_t k = 0; k < s->active.size();) {
    Active &a = s->active[k];
    cudaError_t q = cudaEventQuery(a.done);
    if (q == cudaErrorNotReady) {
      k++;
      continue;
    }
    if (q != cudaSuccess) {
      cudaGetLastError();
      retire(s, k, IBM_ECUDA);
      continue;
    }
    if (a.launched >= a.req->nsteps) {
      retire(s, k, IBM_OK);
      continue;
    }
    k++;
  }
  // admit waiting requests, in arrival order, while a slot and memory are free
  while (!s->pending.empty() && (int)s->active.size() < s->max_active && s->used + s->pending.front()->bytes <= s->budget) {
    Request *r = s->pending.front();
    s->pending.pop_front();
    Active a{};
    a.req = r;
    cudaError_t e = cudaStreamCreateWithFlags(&a.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming);
    ibm_status st = e == cudaSuccess ? ibm_create_case(&r->geo, &r->grid, &r->flow, &r->motion, a.stream, &a.c)
                                     : IBM_ECUDA;
    if (st == IBM_OK) st = ibm_classify(a.c);
    if (st != IBM_OK) {
      cudaGetLastError();
      if (a.c) ibm_destroy_case(a.c);
      if (a.done) cudaEventDestroy(a.done);
      if (a.stream) cudaStreamDestroy(a.stream);
      r->res.status = st;
      r->res.state = IBM_REQ_FAILED;
      r->res.finish_s = now_s(s->t0);
      continue;
    }
    r->res.state = IBM_REQ_RUNNING;
    r->res.start_s = now_s(s->t0);
    s->used += r->bytes;
    cudaEventRecord(a.done, a.stream);
    s->active.push_back(a);
  }
  // enqueue the next chunk of steps of every case whose previous chunk is done
  for (Active &a : s->active) {
    if (a.launched >= a.req->nsteps) continue;
    if (cudaEventQuery(a.done) == cudaErrorNotReady) continue;
    const int n = a.req->nsteps - a.launched < s->chunk ? a.req->nsteps - a.launched : s->chunk;
    ibm_status st = ibm_step(a.c, n);
    if (st != IBM_OK) {
      a.launched = a.req->nsteps;  // retired (as failed) on the next round
      a.req->res.status = st;
    } else {
      a.launched += n;
    }
    cudaEventRecord(a.done, a.stream);
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
  while (!s->active.empty()) {
    cudaStreamSynchronize(s->active.back().stream);
    retire(s, s->active.size() - 1, IBM_ESTATE);
  }
  for (auto &kv : s->all) delete kv.second;
  delete s;
  return IBM_OK;
}
