// Admission and scheduling core of the merge server (host only, no CUDA).
//
// Requests to merge a registered table arrive over time.  A request is
// admitted when (1) a slot (one concurrent table merge) is free, (2) its
// table has no merge in flight (a table's output buffers serve one merge
// at a time) and is not paused, and (3) a contiguous region of its HBM
// footprint fits the scratch pool (first fit).  Queued requests are
// scanned in arrival order and any admissible one starts (a request
// blocked by a busy or paused table does not hold back the others), so new
// work joins as soon as slots and memory free up: continuous batching.
// Completion frees the region and the slot and commits the table's new
// version.
//
// Online tables (Section 3 of the paper) take inserts while they serve
// merges.  Each has two delta partitions: inserts append to the active
// one; when a merge of the table is admitted, the active delta is frozen
// (the merge works on the committed main plus that delta) and the other,
// empty one becomes active, so rows inserted during the merge collect in a
// second delta; the commit at completion makes the merged main the table's
// main, empties the frozen delta, and the second delta is then the one the
// next merge takes.  A merge is requested automatically once the active
// delta holds more than a fraction k of the main's rows (Section 4's
// trigger N_D > k N_M); pausing a table holds its merges back (Section 3:
// a scheduler may pause and resume the merge) while inserts go on.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

namespace dm {

class ScratchPool {
 public:
  explicit ScratchPool(uint64_t bytes) : size_(bytes) {
    if (bytes) free_[0] = bytes;
  }
  static constexpr uint64_t kAlign = 256;
  // First-fit allocation; returns false when no free run is long enough.
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    if (bytes == 0) bytes = kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    if (bytes == 0) bytes = kAlign;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t used() const { return used_; }
  uint64_t size() const { return size_; }

 private:
  uint64_t size_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;   // offset -> length
};

struct SchedRequest {
  uint64_t id = 0;
  uint32_t table = 0;
  uint64_t submit_ns = 0, admit_ns = 0, done_ns = 0;
  uint64_t footprint = 0, offset = 0;
  uint32_t slot = 0;
  int status = 0;
  bool admitted = false, done = false;
  bool automatic = false;     // requested by the online trigger
  // online tables: the delta the merge took and its rows, the version it
  // commits (0 for a merge that found no rows: nothing is committed)
  uint32_t delta = 0;
  uint64_t delta_rows = 0;
  uint64_t version = 0;
  uint64_t digest = 0;        // checksum of the merge's outputs (when the server computes one)
  uint64_t tuples = 0;        // online tables: tuple-columns the merge covers
};

// Where an insert into an online table went.
struct SchedInsert {
  int status = 0;             // 0 ok, 1 no such online table, 2 a delta or a capacity is full
  uint32_t delta = 0;         // delta partition (0 or 1) the rows were appended to
  uint64_t first_row = 0;     // their first row in it
  uint64_t lands_in = 0;      // version of the table that will contain them
  bool triggered = false;     // the insert requested a merge
  uint64_t request = 0;       // that request
};

struct SchedAdmit {
  uint64_t request;
  uint32_t slot;
  uint64_t offset, bytes;
};

class Scheduler {
 public:
  Scheduler(uint64_t pool_bytes, uint32_t slots) : pool_(pool_bytes), slot_busy_(slots, false) {}

  // false when the table alone cannot fit the pool
  bool add_table(uint32_t id, uint64_t footprint) {
    if (footprint > pool_.size()) return false;
    Table t;
    t.footprint = footprint;
    tables_[id] = t;
    return true;
  }
  // An online table of main_rows rows whose deltas hold delta_cap rows each
  // and whose main may grow to rows_cap rows; trigger k > 0 requests a merge
  // once the active delta holds more than k * main_rows rows (0: merges only
  // on request).
  bool add_online_table(uint32_t id, uint64_t footprint, uint64_t main_rows, uint64_t rows_cap,
                        uint64_t delta_cap, double trigger) {
    if (!add_table(id, footprint)) return false;
    Table& t = tables_[id];
    t.online = true;
    t.main_rows = main_rows;
    t.rows_cap = rows_cap;
    t.delta_cap = delta_cap;
    t.trigger = trigger;
    return true;
  }
  bool has_table(uint32_t id) const { return tables_.count(id) != 0; }
  bool is_online(uint32_t id) const {
    auto it = tables_.find(id);
    return it != tables_.end() && it->second.online;
  }

  uint64_t submit(uint32_t table, uint64_t now, bool automatic = false) {
    SchedRequest r;
    r.id = reqs_.size();
    r.table = table;
    r.submit_ns = now;
    r.footprint = tables_.at(table).footprint;
    r.automatic = automatic;
    reqs_.push_back(r);
    queue_.push_back(r.id);
    ++tables_.at(table).queued;
    return r.id;
  }

  // Append `rows` rows to the online table's active delta (all of them or
  // none: status 2 when the delta or the main's row capacity would be
  // exceeded); requests a merge when the trigger fires and none is queued.
  SchedInsert insert(uint32_t table, uint64_t rows, uint64_t now) {
    SchedInsert out;
    auto it = tables_.find(table);
    if (it == tables_.end() || !it->second.online) {
      out.status = 1;
      return out;
    }
    Table& t = it->second;
    const uint64_t pending = t.delta_rows[0] + t.delta_rows[1];
    if (t.delta_rows[t.active] + rows > t.delta_cap || t.main_rows + pending + rows > t.rows_cap) {
      out.status = 2;
      return out;
    }
    out.delta = t.active;
    out.first_row = t.delta_rows[t.active];
    t.delta_rows[t.active] += rows;
    // a merge in flight (or one to retry) holds the other delta: these
    // rows come one version after it
    out.lands_in = t.version + 1 + (t.frozen != kNone && t.delta_rows[t.frozen] ? 1 : 0);
    if (want_merge(t)) {
      out.triggered = true;
      out.request = submit(table, now, true);
    }
    return out;
  }

  // Merges of a paused table are not admitted (queued ones wait, the
  // trigger still queues them); resume lets them start.
  bool set_paused(uint32_t table, bool paused) {
    auto it = tables_.find(table);
    if (it == tables_.end()) return false;
    it->second.paused = paused;
    return true;
  }
  bool paused(uint32_t table) const { return tables_.at(table).paused; }

  // Requests that start now (arrival order, skipping the blocked ones).
  std::vector<SchedAdmit> admit(uint64_t now) {
    std::vector<SchedAdmit> out;
    for (auto it = queue_.begin(); it != queue_.end();) {
      const uint32_t slot = free_slot();
      if (slot == kNone) break;
      SchedRequest& r = reqs_[*it];
      Table& t = tables_.at(r.table);
      uint64_t off = 0;
      if (t.busy || t.paused || !pool_.alloc(r.footprint, &off)) {
        ++it;
        continue;
      }
      t.busy = true;
      --t.queued;
      slot_busy_[slot] = true;
      r.admitted = true;
      r.admit_ns = now;
      r.offset = off;
      r.slot = slot;
      if (t.online) {
        // freeze the active delta (a merge that failed before keeps its
        // frozen delta and takes it again); inserts now go to the other one
        if (t.frozen == kNone) {
          t.frozen = t.active;
          t.active ^= 1u;
        }
        r.delta = t.frozen;
        r.delta_rows = t.delta_rows[t.frozen];
      }
      inflight_ += r.footprint;
      ++running_;
      peak_bytes_ = std::max(peak_bytes_, pool_.used());
      peak_running_ = std::max(peak_running_, running_);
      out.push_back({r.id, slot, off, r.footprint});
      it = queue_.erase(it);
    }
    return out;
  }

  // The request finished (status 0 = ok); frees its slot and region and
  // commits its table's new version.  For an online table the merged rows
  // join the main and their delta empties; when the active delta is past
  // the trigger by then, the next merge is requested at once (its id in
  // *triggered, else kNoRequest).
  void complete(uint64_t id, uint64_t now, int status, uint64_t* triggered = nullptr) {
    SchedRequest& r = reqs_[id];
    r.done = true;
    r.done_ns = now;
    r.status = status;
    Table& t = tables_.at(r.table);
    t.busy = false;
    if (t.online) {
      if (status == 0) {
        if (r.delta_rows) {
          t.main_rows += r.delta_rows;
          ++t.version;
          r.version = t.version;
        }
        t.delta_rows[t.frozen] = 0;
        t.frozen = kNone;
      }
    } else if (status == 0) {
      ++t.version;
      r.version = t.version;
    }
    slot_busy_[r.slot] = false;
    pool_.release(r.offset, r.footprint);
    inflight_ -= r.footprint;
    --running_;
    if (triggered) *triggered = kNoRequest;
    if (t.online && want_merge(t)) {
      const uint64_t q = submit(r.table, now, true);
      if (triggered) *triggered = q;
    }
  }

  bool idle() const { return queue_.empty() && running_ == 0; }
  uint32_t running() const { return running_; }
  uint64_t peak_bytes() const { return peak_bytes_; }
  uint32_t peak_running() const { return peak_running_; }
  uint64_t version(uint32_t table) const { return tables_.at(table).version; }
  const std::vector<SchedRequest>& requests() const { return reqs_; }
  std::vector<SchedRequest>& requests_mut() { return reqs_; }
  uint64_t pool_bytes() const { return pool_.size(); }
  // online tables: rows of the committed main, and of each delta
  uint64_t main_rows(uint32_t table) const { return tables_.at(table).main_rows; }
  uint64_t delta_rows(uint32_t table, uint32_t k) const { return tables_.at(table).delta_rows[k & 1]; }
  uint32_t active_delta(uint32_t table) const { return tables_.at(table).active; }

  static constexpr uint64_t kNoRequest = ~0ull;

 private:
  static constexpr uint32_t kNone = 0xFFFFFFFFu;
  struct Table {
    uint64_t footprint = 0;
    bool busy = false;
    uint64_t version = 0;
    bool paused = false;
    uint32_t queued = 0;        // requests of the table waiting for admission
    // online tables
    bool online = false;
    uint64_t main_rows = 0, rows_cap = 0, delta_cap = 0;
    uint64_t delta_rows[2] = {0, 0};
    uint32_t active = 0;        // delta receiving inserts
    uint32_t frozen = kNone;    // delta taken by the merge in flight (or to retry)
    double trigger = 0;
  };
  // The online trigger: active delta past k * N_M, no merge of the table
  // queued, and none in flight (a merge in flight re-checks at its commit).
  static bool want_merge(const Table& t) {
    return t.trigger > 0 && t.queued == 0 && !t.busy &&
           (double)t.delta_rows[t.active] > t.trigger * (double)t.main_rows;
  }
  uint32_t free_slot() const {
    for (uint32_t i = 0; i < slot_busy_.size(); ++i)
      if (!slot_busy_[i]) return i;
    return kNone;
  }
  ScratchPool pool_;
  std::vector<bool> slot_busy_;
  std::unordered_map<uint32_t, Table> tables_;
  std::vector<SchedRequest> reqs_;
  std::deque<uint64_t> queue_;
  uint64_t inflight_ = 0, peak_bytes_ = 0;
  uint32_t running_ = 0, peak_running_ = 0;
};

}  // namespace dm
