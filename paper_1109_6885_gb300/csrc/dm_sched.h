// Admission and scheduling core of the merge server (host only, no CUDA).
//
// Requests to merge a registered table arrive over time.  A request is
// admitted when (1) a slot (one concurrent table merge) is free, (2) its
// table has no merge in flight (a table's output buffers serve one merge
// at a time), and (3) a contiguous region of its HBM footprint fits the
// scratch pool (first fit).  Queued requests are scanned in arrival order
// and any admissible one starts (a request blocked by a busy table does
// not hold back the others), so new work joins as soon as slots and memory
// free up: continuous batching.  Completion frees the region and the slot
// and commits the table's new version.
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
    tables_[id] = Table{footprint, false, 0};
    return true;
  }
  bool has_table(uint32_t id) const { return tables_.count(id) != 0; }

  uint64_t submit(uint32_t table, uint64_t now) {
    SchedRequest r;
    r.id = reqs_.size();
    r.table = table;
    r.submit_ns = now;
    r.footprint = tables_.at(table).footprint;
    reqs_.push_back(r);
    queue_.push_back(r.id);
    return r.id;
  }

  // Requests that start now (arrival order, skipping the blocked ones).
  std::vector<SchedAdmit> admit(uint64_t now) {
    std::vector<SchedAdmit> out;
    for (auto it = queue_.begin(); it != queue_.end();) {
      const uint32_t slot = free_slot();
      if (slot == kNone) break;
      SchedRequest& r = reqs_[*it];
      Table& t = tables_.at(r.table);
      uint64_t off = 0;
      if (t.busy || !pool_.alloc(r.footprint, &off)) {
        ++it;
        continue;
      }
      t.busy = true;
      slot_busy_[slot] = true;
      r.admitted = true;
      r.admit_ns = now;
      r.offset = off;
      r.slot = slot;
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
  // commits its table's new version.
  void complete(uint64_t id, uint64_t now, int status) {
    SchedRequest& r = reqs_[id];
    r.done = true;
    r.done_ns = now;
    r.status = status;
    Table& t = tables_.at(r.table);
    t.busy = false;
    if (status == 0) ++t.version;
    slot_busy_[r.slot] = false;
    pool_.release(r.offset, r.footprint);
    inflight_ -= r.footprint;
    --running_;
  }

  bool idle() const { return queue_.empty() && running_ == 0; }
  uint32_t running() const { return running_; }
  uint64_t peak_bytes() const { return peak_bytes_; }
  uint32_t peak_running() const { return peak_running_; }
  uint64_t version(uint32_t table) const { return tables_.at(table).version; }
  const std::vector<SchedRequest>& requests() const { return reqs_; }
  uint64_t pool_bytes() const { return pool_.size(); }

 private:
  static constexpr uint32_t kNone = 0xFFFFFFFFu;
  struct Table {
    uint64_t footprint;
    bool busy;
    uint64_t version;
  };
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
