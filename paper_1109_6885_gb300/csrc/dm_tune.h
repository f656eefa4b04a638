// Tune cache behind the opaque dm_tune_cache handle (internal, host only).
//
// Maps a column class (dm_tune_key) to the launch choices measured fastest
// for it (dm_tune_choice).  Every choice gives the same output bytes; the
// cache only changes how the work is split.  Thread-safe: server slots on
// several host threads may share one cache.
#pragma once

#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dmerge.h"

struct dm_tune_cache {
  using Key = std::tuple<uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;
  mutable std::mutex mu;
  std::map<Key, dm_tune_choice> entries;
  uint64_t generation = 0;   // bumped by every change, so cached table graphs notice
  std::atomic<uint64_t> size{0};   // entries.size(), readable without the lock

  static Key key_of(const dm_tune_key& k) {
    return Key{k.value_bytes, k.main_bits, k.max_bits, k.log2_m, k.log2_d, k.log2_main_rows,
               k.log2_delta_rows};
  }
};

namespace dm {

// A choice the library accepts (fields in range; 0 = default everywhere).
bool tune_choice_valid(const dm_tune_choice& c);
// Class of a column: bit lengths of its sizes, its width and input bits.
dm_tune_key tune_key_of(const dm_column_in& in);
// Entries as the text of a JSON document, and back (false: malformed).
std::string tune_cache_to_json(const dm_tune_cache& c);
bool tune_cache_from_json(const std::string& text, std::vector<std::pair<dm_tune_key, dm_tune_choice>>* out);

}  // namespace dm
