// serve.cpp -- a serving engine for conjunctive queries over a resident
// index: continuous batching on the device.
//
// The caller hands over the index (device data + descriptors), `slots`
// CUDA streams, one device buffer and one pinned host buffer.  Each slot
// owns a fixed slice of both.  Queries are submitted from any host thread
// and wait in an arrival queue.  A dispatcher thread repeatedly
//   - moves on slots whose batch has finished on the device: the kernels
//     wrote the answers to the slot's device memory and the counts and
//     offsets straight into its pinned host memory, so the exact number of
//     answer values is known and one copy-engine transfer brings them to
//     the slot's pinned memory (kernel stores over the host link measured
//     58 GB/s, half what this needs at the device's query rate; the copy
//     engines move about 190 GB/s);
//   - retires slots whose transfer has finished, stamping each query's
//     completion time, and
//   - admits waiting queries into every free slot, in arrival order, as long
//     as the batch's scratch and answer capacity fit the slot's memory, and
//     launches bp_query_batch for them on the slot's stream.
// So requests that arrive while other batches are on the GPU are admitted as
// soon as a slot and its memory are free, and several batches run on the
// device at once.  Nothing here allocates device or pinned memory.
//
// The shared arrival queue is held only for moves: the dispatcher takes
// everything queued into a backlog of its own in one step and sizes batches
// from there, so submitters (up to a million per second) never wait for an
// admission decision.  Each query carries the time it was due (its scheduled
// arrival under replay) besides the time it was queued, and latency counts
// from the former.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bp128.h"
#include "decode.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

inline size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Pending {
  uint64_t tag;
  double arrival_s, submit_s;
  uint32_t k;
  uint32_t terms[64];
};

struct Done {
  uint64_t tag;
  uint32_t count;
  int32_t status;
  double arrival_s, submit_s, done_s;
  std::vector<uint32_t> answer;
};

constexpr size_t kBatchRecords = 1u << 20;  // timeline entries kept

struct Slot {
  cudaStream_t stream;
  cudaEvent_t ev;
  bool busy = false;
  bool copying = false;  // the answers are on their way to pinned memory
  // device slice
  uint8_t *d_base;
  uint32_t *d_terms;
  uint64_t *d_toff;
  uint32_t *d_status;
  uint8_t *d_scratch;
  // pinned host slice (device-accessible)
  uint8_t *h_base;
  uint32_t *h_terms;
  uint64_t *h_toff;
  uint64_t *h_out_off;
  uint32_t *h_counts;
  uint32_t *h_status;
  uint32_t *h_answers;
  // the batch in flight
  std::vector<Pending> batch;
  uint64_t out_cap = 0;
  bp_server_batch rec{};
};

}  // namespace

struct bp_server {
  bp_server_config cfg;
  const uint8_t *d_data;
  const bp_list *d_lists;
  std::vector<bp_list> h_lists;
  uint32_t n_terms;
  int device;
  std::vector<Slot> slots;
  size_t fixed_dev, fixed_host, slot_dev, slot_host;

  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> queue;    // shared with the submitters (under mu)
  std::deque<Pending> backlog;  // the dispatcher's own, in arrival order
  std::atomic<uint64_t> backlog_size{0};
  std::deque<Done> done;
  std::vector<Done> polled;  // answers handed out by the last poll
  std::deque<bp_server_batch> records;  // retired batches (under mu)
  uint64_t submitted = 0, completed = 0, batches = 0, rejected = 0, max_busy = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  int first_error = BP_OK;

  void run();
  void take_arrivals();
  bool admit(Slot &s, uint32_t slot_index);
  void retire(Slot &s);
  int submit_at(uint64_t tag, const uint32_t *terms, uint32_t k, double arrival_s);
};

namespace {

// Fixed part of a slot: term ids, term offsets, status (device) and the
// matching pinned copies plus counts and offsets.
void slot_layout(const bp_server_config &c, size_t &fixed_dev, size_t &fixed_host) {
  const size_t terms = up256(4ull * c.max_batch_queries * c.max_terms);
  const size_t toff = up256(8ull * (c.max_batch_queries + 1));
  fixed_dev = terms + toff + 256;
  fixed_host = terms + toff + toff + up256(4ull * c.max_batch_queries) + 256;
}

}  // namespace

void bp_server::take_arrivals() {
  std::lock_guard<std::mutex> g(mu);
  if (queue.empty()) return;
  if (backlog.empty()) {
    backlog.swap(queue);
  } else {
    for (auto &p : queue) backlog.push_back(p);
    queue.clear();
  }
  backlog_size.store(backlog.size());
}

bool bp_server::admit(Slot &s, uint32_t slot_index) {
  // take queries from the head of the backlog while they fit the slot
  const double t_admit = now_s();
  std::vector<Pending> take;
  std::vector<Done> rejects;
  std::vector<uint32_t> terms;
  std::vector<uint64_t> toff(1, 0);
  uint64_t cap = 0, items = 0;
  while (!backlog.empty() && take.size() < cfg.max_batch_queries) {
    const Pending &p = backlog.front();
    uint64_t nmin = 0, qitems = 0;
    if (p.k) {
      nmin = UINT64_MAX;
      const bp_list *drv = &h_lists[p.terms[0]];
      for (uint32_t i = 0; i < p.k; i++) {
        const bp_list &L = h_lists[p.terms[i]];
        nmin = std::min<uint64_t>(nmin, L.n);
        // the list that drives the query: compressed before bitmaps, then shortest
        const bool lb = L.layout == BP_LAYOUT_BITMAP, db = drv->layout == BP_LAYOUT_BITMAP;
        if (lb < db || (lb == db && L.n < drv->n)) drv = &L;
      }
      qitems = bp::query_items_of(*drv);
    }
    // memory this batch would need with p added
    const uint64_t cap2 = cap + nmin, items2 = items + qitems;
    const size_t need = bp::query_batch_scratch_for(terms.size() + p.k, (uint32_t)take.size() + 1,
                                                    std::max<uint64_t>(cap2, 1), items2);
    const bool fits_dev =  // answers, then scratch
        need + up256(4 * std::max<uint64_t>(cap2, 1)) <= slot_dev - fixed_dev;
    const bool fits_host = 4 * cap2 <= slot_host - fixed_host;
    if (!fits_dev || !fits_host) {
      if (take.empty()) {  // can never fit this slot: reject it
        rejects.push_back(Done{p.tag, 0, BP_ERR_SCRATCH, p.arrival_s, p.submit_s, now_s(), {}});
        backlog.pop_front();
        continue;
      }
      break;
    }
    terms.insert(terms.end(), p.terms, p.terms + p.k);
    toff.push_back(toff.back() + p.k);
    cap = cap2;
    items = items2;
    take.push_back(p);
    backlog.pop_front();
  }
  backlog_size.store(backlog.size());
  if (!rejects.empty()) {
    std::lock_guard<std::mutex> g(mu);
    for (auto &d : rejects) done.push_back(std::move(d));
    rejected += rejects.size();
    completed += rejects.size();
  }
  if (take.empty()) return !rejects.empty();
  const uint32_t nq = (uint32_t)take.size();
  std::memcpy(s.h_terms, terms.data(), 4 * terms.size());
  std::memcpy(s.h_toff, toff.data(), 8 * toff.size());
  cudaStream_t st = s.stream;
  int rc = BP_OK;
  if (terms.size() &&
      cudaMemcpyAsync(s.d_terms, s.h_terms, 4 * terms.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    rc = BP_ERR_CUDA;
  if (rc == BP_OK &&
      (cudaMemcpyAsync(s.d_toff, s.h_toff, 8 * toff.size(), cudaMemcpyHostToDevice, st) !=
           cudaSuccess ||
       cudaMemsetAsync(s.d_status, 0, 4, st) != cudaSuccess))
    rc = BP_ERR_CUDA;
  // the answers go to the front of the slot's device memory, the scratch
  // after them; counts and offsets straight to pinned memory
  const uint64_t out_cap = std::max<uint64_t>(cap, 1);
  const size_t ans_bytes = up256(4 * out_cap);
  if (rc == BP_OK)
    rc = bp::launch_query_batch(d_data, d_lists, n_terms, s.d_terms, s.d_toff, terms.size(), nq,
                                reinterpret_cast<uint32_t *>(s.d_scratch), out_cap, s.h_out_off,
                                s.h_counts, s.d_scratch + ans_bytes,
                                slot_dev - fixed_dev - ans_bytes, s.d_status, st);
  if (rc == BP_OK &&
      (cudaMemcpyAsync(s.h_status, s.d_status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaEventRecord(s.ev, st) != cudaSuccess))
    rc = BP_ERR_CUDA;
  double first_arrival = take.front().arrival_s;
  for (const auto &p : take) first_arrival = std::min(first_arrival, p.arrival_s);
  s.rec = bp_server_batch{slot_index, nq, 0, first_arrival, t_admit, now_s(), 0.0, 0.0};
  s.batch.swap(take);
  s.out_cap = out_cap;
  s.busy = true;
  batches++;
  if (rc != BP_OK) {  // report the launch failure on every query of the batch
    const double t = now_s();
    std::lock_guard<std::mutex> g(mu);
    if (first_error == BP_OK) first_error = rc;
    for (auto &p : s.batch) done.push_back(Done{p.tag, 0, rc, p.arrival_s, p.submit_s, t, {}});
    completed += s.batch.size();
    s.batch.clear();
    s.busy = false;
  }
  return true;
}

void bp_server::retire(Slot &s) {
  const double t = now_s();
  const int st = (int)*s.h_status;
  std::vector<Done> out;
  out.reserve(s.batch.size());
  uint64_t values = 0;
  for (size_t q = 0; q < s.batch.size(); q++) {
    const Pending &p = s.batch[q];
    Done d{p.tag, s.h_counts[q], st, p.arrival_s, p.submit_s, t, {}};
    values += d.count;
    if (cfg.deliver_answers && st == BP_OK) {
      const uint64_t o = s.h_out_off[q];
      d.answer.assign(s.h_answers + o, s.h_answers + o + d.count);
    }
    out.push_back(std::move(d));
  }
  s.rec.answer_values = values;
  if (s.rec.done_s == 0.0) s.rec.done_s = t;
  s.rec.retired_s = now_s();
  s.copying = false;
  {
    std::lock_guard<std::mutex> g(mu);
    for (auto &d : out) done.push_back(std::move(d));
    completed += s.batch.size();
    if (st != BP_OK && first_error == BP_OK) first_error = st;
    if (records.size() >= kBatchRecords) records.pop_front();
    records.push_back(s.rec);
  }
  s.batch.clear();
  s.busy = false;
}

void bp_server::run() {
  cudaSetDevice(device);
  while (true) {
    bool worked = false;
    for (auto &s : slots) {
      if (!s.busy || cudaEventQuery(s.ev) != cudaSuccess) continue;
      worked = true;
      if (!s.copying) {  // the batch is done on the device: bring its answers over
        s.rec.done_s = now_s();
        const uint64_t total = s.h_out_off[s.batch.size()];
        if ((int)*s.h_status == BP_OK && total > 0 && total <= s.out_cap) {
          if (cudaMemcpyAsync(s.h_answers, s.d_scratch, 4 * total, cudaMemcpyDeviceToHost,
                              s.stream) == cudaSuccess &&
              cudaEventRecord(s.ev, s.stream) == cudaSuccess) {
            s.copying = true;
            continue;
          }
          *s.h_status = BP_ERR_CUDA;
        }
      }
      retire(s);
    }
    take_arrivals();
    for (uint32_t i = 0; i < slots.size(); i++)
      if (!slots[i].busy && admit(slots[i], i)) worked = true;
    uint64_t busy = 0;
    for (auto &s : slots) busy += s.busy ? 1 : 0;
    if (busy > max_busy) {
      std::lock_guard<std::mutex> g(mu);
      max_busy = busy;
    }
    if (stop.load() && !worked) {
      bool idle = backlog.empty();
      for (auto &s : slots) idle &= !s.busy;
      std::lock_guard<std::mutex> g(mu);
      if (idle && queue.empty()) break;
    }
    if (!worked) {
      std::unique_lock<std::mutex> lk(mu);
      if (queue.empty()) cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

int bp_server::submit_at(uint64_t tag, const uint32_t *terms, uint32_t k, double arrival_s) {
  if ((k && !terms) || k > cfg.max_terms) return BP_ERR_ARG;
  for (uint32_t i = 0; i < k; i++)
    if (terms[i] >= n_terms) return BP_ERR_ARG;
  Pending p;
  p.tag = tag;
  p.k = k;
  std::memcpy(p.terms, terms, 4ull * k);
  p.submit_s = now_s();
  p.arrival_s = arrival_s > 0.0 ? arrival_s : p.submit_s;
  {
    std::lock_guard<std::mutex> g(mu);
    queue.push_back(p);
    submitted++;
  }
  cv.notify_one();
  return BP_OK;
}

extern "C" {

size_t bp_server_device_bytes(const bp_server_config *cfg) {
  return cfg ? (size_t)cfg->slots * cfg->slot_bytes : 0;
}

size_t bp_server_host_bytes(const bp_server_config *cfg) {
  if (!cfg) return 0;
  size_t fd, fh;
  slot_layout(*cfg, fd, fh);
  return (size_t)cfg->slots * (fh + up256(cfg->slot_bytes));
}

bp_server *bp_server_create(const uint8_t *d_data, const bp_list *d_lists, const bp_list *h_lists,
                            uint32_t n_terms, const bp_server_config *cfg, void *d_mem,
                            void *h_pinned, void *const *streams, int *err) {
  auto fail = [&](int code) -> bp_server * {
    if (err) *err = code;
    return nullptr;
  };
  if (!d_data || !d_lists || !h_lists || !cfg || !d_mem || !h_pinned || !streams)
    return fail(BP_ERR_ARG);
  if (cfg->slots < 1 || cfg->slots > 16 || cfg->max_batch_queries < 1 || cfg->max_terms < 1 ||
      cfg->max_terms > 64)
    return fail(BP_ERR_ARG);
  size_t fd, fh;
  slot_layout(*cfg, fd, fh);
  if (cfg->slot_bytes <= fd + 4096) return fail(BP_ERR_SCRATCH);
  // the answers are written by the kernels straight into the pinned buffer
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, h_pinned) != cudaSuccess || pa.devicePointer == nullptr ||
      pa.devicePointer != h_pinned)
    return fail(BP_ERR_ARG);
  auto *s = new bp_server();
  s->cfg = *cfg;
  s->d_data = d_data;
  s->d_lists = d_lists;
  s->h_lists.assign(h_lists, h_lists + n_terms);
  s->n_terms = n_terms;
  cudaGetDevice(&s->device);
  s->fixed_dev = fd;
  s->fixed_host = fh;
  s->slot_dev = cfg->slot_bytes;
  s->slot_host = fh + up256(cfg->slot_bytes);
  s->slots.resize(cfg->slots);
  for (uint32_t i = 0; i < cfg->slots; i++) {
    Slot &sl = s->slots[i];
    sl.stream = static_cast<cudaStream_t>(streams[i]);
    if (cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      delete s;
      return fail(BP_ERR_CUDA);
    }
    const size_t terms = up256(4ull * cfg->max_batch_queries * cfg->max_terms);
    const size_t toff = up256(8ull * (cfg->max_batch_queries + 1));
    uint8_t *d = static_cast<uint8_t *>(d_mem) + (size_t)i * cfg->slot_bytes;
    sl.d_base = d;
    sl.d_terms = reinterpret_cast<uint32_t *>(d);
    sl.d_toff = reinterpret_cast<uint64_t *>(d + terms);
    sl.d_status = reinterpret_cast<uint32_t *>(d + terms + toff);
    sl.d_scratch = d + fd;
    uint8_t *h = static_cast<uint8_t *>(h_pinned) + (size_t)i * s->slot_host;
    sl.h_base = h;
    sl.h_terms = reinterpret_cast<uint32_t *>(h);
    sl.h_toff = reinterpret_cast<uint64_t *>(h + terms);
    sl.h_out_off = reinterpret_cast<uint64_t *>(h + terms + toff);
    sl.h_counts = reinterpret_cast<uint32_t *>(h + terms + 2 * toff);
    sl.h_status = reinterpret_cast<uint32_t *>(h + terms + 2 * toff +
                                               up256(4ull * cfg->max_batch_queries));
    sl.h_answers = reinterpret_cast<uint32_t *>(h + fh);
  }
  s->worker = std::thread([s] { s->run(); });
  if (err) *err = BP_OK;
  return s;
}

int bp_server_submit(bp_server *s, uint64_t tag, const uint32_t *terms, uint32_t k) {
  if (!s) return BP_ERR_ARG;
  return s->submit_at(tag, terms, k, 0.0);
}

int bp_server_replay(bp_server *s, const uint64_t *tags, const uint32_t *terms,
                     const uint64_t *term_off, uint32_t n, const double *arrival_s) {
  if (!s || !tags || !term_off || !arrival_s) return BP_ERR_ARG;
  const double t0 = now_s();
  for (uint32_t i = 0; i < n; i++) {
    const double due = t0 + arrival_s[i];
    while (now_s() < due) {
    }
    const int rc = s->submit_at(tags[i], terms + term_off[i],
                                (uint32_t)(term_off[i + 1] - term_off[i]), due);
    if (rc != BP_OK) return rc;
  }
  return BP_OK;
}

uint32_t bp_server_poll(bp_server *s, bp_server_result *out, uint32_t max) {
  if (!s || !out) return 0;
  std::lock_guard<std::mutex> g(s->mu);
  s->polled.clear();
  uint32_t n = 0;
  while (n < max && !s->done.empty()) {
    s->polled.push_back(std::move(s->done.front()));
    s->done.pop_front();
    n++;
  }
  for (uint32_t i = 0; i < n; i++) {
    const Done &d = s->polled[i];
    out[i].tag = d.tag;
    out[i].count = d.count;
    out[i].status = d.status;
    out[i].arrival_s = d.arrival_s;
    out[i].submit_s = d.submit_s;
    out[i].done_s = d.done_s;
    out[i].answer = d.answer.empty() ? nullptr : d.answer.data();
  }
  return n;
}

int bp_server_drain(bp_server *s, double timeout_s) {
  if (!s) return BP_ERR_ARG;
  const double t_end = now_s() + timeout_s;
  while (now_s() < t_end) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      if (s->completed == s->submitted) return s->first_error;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  return BP_ERR_TIMEOUT;
}

int bp_server_stats(bp_server *s, uint64_t out[6]) {
  if (!s || !out) return BP_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  out[0] = s->submitted;
  out[1] = s->completed;
  out[2] = s->batches;
  out[3] = s->rejected;
  out[4] = s->max_busy;
  out[5] = s->queue.size() + s->backlog_size.load();
  return BP_OK;
}

uint32_t bp_server_batches(bp_server *s, bp_server_batch *out, uint32_t max) {
  if (!s || !out) return 0;
  std::lock_guard<std::mutex> g(s->mu);
  uint32_t n = 0;
  while (n < max && !s->records.empty()) {
    out[n++] = s->records.front();
    s->records.pop_front();
  }
  return n;
}

void bp_server_destroy(bp_server *s) {
  if (!s) return;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &sl : s->slots) cudaEventDestroy(sl.ev);
  delete s;
}

}  // extern "C"
