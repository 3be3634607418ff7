// Served form: a request loop around the batched path. Clients open sessions
// (one probe volume each); a session is admitted while its volume fits the
// device-memory budget and a slot is free, otherwise it waits in FIFO order
// and is admitted as soon as closing sessions free enough memory and slots.
// Admitted volumes stay resident. At every tick the clients that submitted
// rays are updated together: their volumes are grouped into batches of equal
// shapes (at most PV_MAX_BATCH each, plans cached until the admitted set
// changes), and each batch runs the batched weights, blend and select/pack
// launches, so the work of every client of a tick shares the same launches
// and overlaps on the device. A ticket names one client's update in one tick;
// pv_poll reports PV_PENDING until that tick's work has completed on the GPU.
#include <stdint.h>
#include <string.h>

#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "pv_internal.h"

namespace {

constexpr size_t kTickWindow = 512;     // ticks whose completion events are kept

struct Client {
  pv_desc desc;
  pv_volume* vol = nullptr;
  uint64_t bytes = 0;
  bool admitted = false;
  bool failed = false;                  // creating its volume failed at admission
  bool submitted = false;               // rays pending for the next tick
  const void* rad = nullptr;
  const void* dist = nullptr;
  const float* dirs = nullptr;
  uint64_t ticket = 0;
  pv_frame frame = {};
};

struct TickRecord {
  uint64_t tick;
  cudaEvent_t done;
};

struct Group {
  std::vector<int> clients;             // client ids, in batch order
  pv_batch* batch = nullptr;
};

using pv_host::DeviceGuard;

bool same_shape(const pv_desc& a, const pv_desc& b) {
  return a.color_interior == b.color_interior && a.vis_interior == b.vis_interior && a.state_fmt == b.state_fmt &&
         a.operand_fmt == b.operand_fmt && a.color_code == b.color_code;
}

}  // namespace

struct pv_server {
  pv_server_desc d;
  int device = 0;
  std::mutex mu;
  uint64_t used = 0;                    // device bytes of the admitted volumes
  int slots = 0;                        // admitted sessions
  std::map<int32_t, Client> clients;    // admitted and waiting sessions
  std::deque<int32_t> waiting;          // FIFO of sessions not yet admitted
  std::vector<Group> groups;            // batches of the current admitted set
  bool groups_dirty = true;
  uint64_t tick = 0;                    // ticks launched so far
  uint64_t next_ticket = 1;
  std::map<uint64_t, std::pair<int32_t, uint64_t>> tickets;   // ticket -> (client, tick)
  std::deque<TickRecord> done;          // completion events of recent ticks
  uint64_t oldest_kept = 0;             // ticks before this one are known complete
};

namespace {

void destroy_groups(pv_server* s) {
  for (Group& g : s->groups)
    if (g.batch) probe_batch_destroy(g.batch);
  s->groups.clear();
  s->groups_dirty = true;
}

// Admits waiting sessions in FIFO order while the head fits.
pv_status admit_waiting(pv_server* s) {
  while (!s->waiting.empty()) {
    const int32_t id = s->waiting.front();
    auto it = s->clients.find(id);
    if (it == s->clients.end()) {
      s->waiting.pop_front();
      continue;
    }
    Client& c = it->second;
    if (s->used + c.bytes > s->d.mem_budget_bytes || s->slots >= s->d.max_slots) break;
    s->waiting.pop_front();
    pv_status st = probe_volume_create(&c.desc, &c.vol);
    if (st != PV_OK) {                   // reported through pv_server_status; the queue moves on
      c.failed = true;
      c.vol = nullptr;
      continue;
    }
    c.admitted = true;
    s->used += c.bytes;
    s->slots += 1;
    s->groups_dirty = true;
  }
  return PV_OK;
}

// Batches of the admitted set: equal shapes, at most max_batch volumes each.
pv_status rebuild_groups(pv_server* s) {
  destroy_groups(s);
  std::vector<int32_t> ids;
  for (auto& kv : s->clients)
    if (kv.second.admitted) ids.push_back(kv.first);
  std::vector<bool> used(ids.size(), false);
  for (size_t i = 0; i < ids.size(); ++i) {
    if (used[i]) continue;
    Group g;
    const pv_desc& a = s->clients[ids[i]].desc;
    for (size_t j = i; j < ids.size() && (int)g.clients.size() < s->d.max_batch; ++j) {
      if (used[j] || !same_shape(a, s->clients[ids[j]].desc)) continue;
      used[j] = true;
      g.clients.push_back(ids[j]);
    }
    s->groups.push_back(g);
  }
  for (Group& g : s->groups) {
    pv_volume* vols[PV_MAX_BATCH];
    for (size_t i = 0; i < g.clients.size(); ++i) vols[i] = s->clients[g.clients[i]].vol;
    pv_status st = probe_batch_create(vols, (int32_t)g.clients.size(), 0, &g.batch);
    if (st != PV_OK) {
      destroy_groups(s);
      return st;
    }
  }
  s->groups_dirty = false;
  return PV_OK;
}

// Forget completion events of old ticks (waiting for them first).
void trim_done(pv_server* s) {
  while (s->done.size() > kTickWindow) {
    TickRecord r = s->done.front();
    cudaEventSynchronize(r.done);
    cudaEventDestroy(r.done);
    s->done.pop_front();
    s->oldest_kept = r.tick + 1;
  }
}

}  // namespace

extern "C" {

pv_status pv_server_create(const pv_server_desc* d, pv_server** out) {
  if (!d || !out) return pv_set_error(PV_ERR_INVALID, "pv_server_create: NULL argument");
  *out = nullptr;
  if (d->max_slots < 1) return pv_set_error(PV_ERR_INVALID, "pv_server_create: max_slots < 1");
  if (d->max_batch < 1 || d->max_batch > PV_MAX_BATCH)
    return pv_set_error(PV_ERR_INVALID, "pv_server_create: max_batch must be 1..%d", PV_MAX_BATCH);
  pv_server* s = new pv_server();
  s->d = *d;
  cudaGetDevice(&s->device);
  *out = s;
  return PV_OK;
}

pv_status pv_server_destroy(pv_server* s) {
  if (!s) return PV_OK;
  DeviceGuard g(s->device);
  for (TickRecord& r : s->done) {
    cudaEventSynchronize(r.done);
    cudaEventDestroy(r.done);
  }
  destroy_groups(s);
  for (auto& kv : s->clients)
    if (kv.second.vol) probe_volume_destroy(kv.second.vol);
  delete s;
  return PV_OK;
}

pv_status pv_server_open(pv_server* s, int32_t client, const pv_desc* desc) {
  if (!s || !desc) return pv_set_error(PV_ERR_INVALID, "pv_server_open: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  DeviceGuard g(s->device);
  if (s->clients.count(client)) return pv_set_error(PV_ERR_INVALID, "pv_server_open: client %d already open", client);
  uint64_t bytes = 0;
  pv_status st = probe_volume_bytes(desc, &bytes);
  if (st != PV_OK) return st;
  if (bytes > s->d.mem_budget_bytes)
    return pv_set_error(PV_ERR_OOM, "pv_server_open: volume needs %llu bytes, budget %llu",
                        (unsigned long long)bytes, (unsigned long long)s->d.mem_budget_bytes);
  Client c;
  c.desc = *desc;
  c.desc.kernel = PV_KERNEL_TCGEN05;
  c.bytes = bytes;
  s->clients[client] = c;
  s->waiting.push_back(client);
  st = admit_waiting(s);
  if (st != PV_OK) return st;
  const Client& a = s->clients[client];
  if (a.failed) {
    s->clients.erase(client);
    return pv_set_error(PV_ERR_OOM, "pv_server_open: creating the volume of client %d failed", client);
  }
  return a.admitted ? PV_OK : PV_PENDING;
}

pv_status pv_server_close(pv_server* s, int32_t client) {
  if (!s) return pv_set_error(PV_ERR_INVALID, "pv_server_close: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  DeviceGuard g(s->device);
  auto it = s->clients.find(client);
  if (it == s->clients.end()) return pv_set_error(PV_ERR_INVALID, "pv_server_close: no client %d", client);
  Client& c = it->second;
  if (c.admitted) {
    // the volume may still be in use by launched ticks
    for (TickRecord& r : s->done) cudaEventSynchronize(r.done);
    destroy_groups(s);
    probe_volume_destroy(c.vol);
    s->used -= c.bytes;
    s->slots -= 1;
  }
  s->clients.erase(it);
  return admit_waiting(s);
}

pv_status pv_server_status(pv_server* s, int32_t client, int32_t* admitted, uint64_t* used_bytes,
                           int32_t* waiting) {
  if (!s) return pv_set_error(PV_ERR_INVALID, "pv_server_status: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (admitted) {
    auto it = s->clients.find(client);
    *admitted = it == s->clients.end() ? -1 : (it->second.admitted ? 1 : (it->second.failed ? -2 : 0));
  }
  if (used_bytes) *used_bytes = s->used;
  if (waiting) *waiting = (int32_t)s->waiting.size();
  return PV_OK;
}

pv_status pv_server_volume(pv_server* s, int32_t client, pv_volume** out) {
  if (!s || !out) return pv_set_error(PV_ERR_INVALID, "pv_server_volume: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->clients.find(client);
  if (it == s->clients.end() || !it->second.admitted)
    return pv_set_error(PV_ERR_INVALID, "pv_server_volume: client %d is not admitted", client);
  *out = it->second.vol;
  return PV_OK;
}

pv_status pv_submit(pv_server* s, int32_t client, const void* radiance, const void* dist, const float* dirs,
                    uint64_t* ticket) {
  if (!s || !radiance || !dist || !dirs || !ticket) return pv_set_error(PV_ERR_INVALID, "pv_submit: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->clients.find(client);
  if (it == s->clients.end()) return pv_set_error(PV_ERR_INVALID, "pv_submit: no client %d", client);
  Client& c = it->second;
  if (!c.admitted) return pv_set_error(PV_ERR_BUSY, "pv_submit: client %d is waiting for admission", client);
  if (c.submitted) return pv_set_error(PV_ERR_BUSY, "pv_submit: client %d already has rays for this tick", client);
  c.rad = radiance;
  c.dist = dist;
  c.dirs = dirs;
  c.submitted = true;
  c.ticket = s->next_ticket++;
  s->tickets[c.ticket] = std::make_pair(client, s->tick);
  *ticket = c.ticket;
  return PV_OK;
}

pv_status pv_server_tick(pv_server* s, void* stream, uint64_t* tick_id) {
  if (!s) return pv_set_error(PV_ERR_INVALID, "pv_server_tick: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  DeviceGuard g(s->device);
  if (s->groups_dirty) {
    pv_status st = rebuild_groups(s);
    if (st != PV_OK) return st;
  }
  for (Group& gr : s->groups) {
    // the submitting clients of this group; a group with a client that did
    // not submit runs only the clients that did, as a smaller batch
    std::vector<int32_t> run;
    for (int32_t id : gr.clients)
      if (s->clients[id].submitted) run.push_back(id);
    if (run.empty()) continue;
    pv_batch* b = gr.batch;
    pv_batch* temp = nullptr;
    if (run.size() != gr.clients.size()) {
      pv_volume* vols[PV_MAX_BATCH];
      for (size_t i = 0; i < run.size(); ++i) vols[i] = s->clients[run[i]].vol;
      pv_status st = probe_batch_create(vols, (int32_t)run.size(), 0, &temp);
      if (st != PV_OK) return st;
      b = temp;
    }
    const void* rad[PV_MAX_BATCH];
    const void* dist[PV_MAX_BATCH];
    const float* dirs[PV_MAX_BATCH];
    for (size_t i = 0; i < run.size(); ++i) {
      const Client& c = s->clients[run[i]];
      rad[i] = c.rad;
      dist[i] = c.dist;
      dirs[i] = c.dirs;
    }
    pv_frame frames[PV_MAX_BATCH];
    pv_status st = probe_batch_update(b, rad, dist, dirs, stream);
    if (st == PV_OK) st = probe_batch_select_and_pack(b, frames, stream);
    if (temp) probe_batch_destroy(temp);
    if (st != PV_OK) return st;
    for (size_t i = 0; i < run.size(); ++i) {
      Client& c = s->clients[run[i]];
      c.frame = frames[i];
      c.submitted = false;
    }
  }
  TickRecord r;
  r.tick = s->tick;
  cudaError_t e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r.done, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return pv_set_error(PV_ERR_CUDA, "pv_server_tick: %s", cudaGetErrorString(e));
  s->done.push_back(r);
  trim_done(s);
  if (tick_id) *tick_id = s->tick;
  s->tick += 1;
  return PV_OK;
}

pv_status pv_poll(pv_server* s, uint64_t ticket, pv_frame* out) {
  if (!s) return pv_set_error(PV_ERR_INVALID, "pv_poll: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return pv_set_error(PV_ERR_INVALID, "pv_poll: unknown ticket %llu", (unsigned long long)ticket);
  const int32_t client = it->second.first;
  const uint64_t tick = it->second.second;
  if (tick >= s->tick) return PV_PENDING;       // its tick has not been launched yet
  if (tick >= s->oldest_kept) {
    const TickRecord& r = s->done[(size_t)(tick - s->oldest_kept)];
    const cudaError_t q = cudaEventQuery(r.done);
    if (q == cudaErrorNotReady) return PV_PENDING;
    if (q != cudaSuccess) return pv_set_error(PV_ERR_CUDA, "pv_poll: %s", cudaGetErrorString(q));
  }
  auto ct = s->clients.find(client);
  if (out && ct != s->clients.end()) *out = ct->second.frame;
  s->tickets.erase(it);
  return PV_OK;
}

}  // extern "C"
