// Tune cache: keys, validation, JSON persistence and the host-only C entry
// points (no device is needed for any of them).
#include "dm_tune.h"

#include <ctype.h>
#include <stdio.h>
#include <string.h>

#include <new>

namespace dm {

namespace {

uint32_t bit_length(uint64_t v) {
  uint32_t n = 0;
  while (v) {
    ++n;
    v >>= 1;
  }
  return n;
}

uint32_t bits_for(uint64_t n) { return n <= 1 ? 0u : bit_length(n - 1); }

// The fields of one entry, by name: the key's first, then the choice's.
struct Field {
  const char* name;
  bool in_key;
  size_t offset;
};
const Field kFields[] = {
    {"w", true, offsetof(dm_tune_key, value_bytes)},
    {"b", true, offsetof(dm_tune_key, main_bits)},
    {"bmax", true, offsetof(dm_tune_key, max_bits)},
    {"lm", true, offsetof(dm_tune_key, log2_m)},
    {"ld", true, offsetof(dm_tune_key, log2_d)},
    {"lnm", true, offsetof(dm_tune_key, log2_main_rows)},
    {"lnd", true, offsetof(dm_tune_key, log2_delta_rows)},
    {"warps", false, offsetof(dm_tune_choice, reencode_warps)},
    {"stages", false, offsetof(dm_tune_choice, reencode_stages)},
    {"obufs", false, offsetof(dm_tune_choice, reencode_obufs)},
    {"staging", false, offsetof(dm_tune_choice, x_staging)},
    {"x8", false, offsetof(dm_tune_choice, x8)},
    {"step1_blocks", false, offsetof(dm_tune_choice, step1_blocks)},
};
constexpr size_t kNumFields = sizeof(kFields) / sizeof(kFields[0]);

uint32_t* field_ptr(const Field& f, dm_tune_key* k, dm_tune_choice* c) {
  char* base = f.in_key ? reinterpret_cast<char*>(k) : reinterpret_cast<char*>(c);
  return reinterpret_cast<uint32_t*>(base + f.offset);
}

// Minimal reader for the document tune_cache_to_json writes: an object
// whose "entries" member is an array of flat objects of unsigned integers.
struct Reader {
  const char* p;
  const char* end;
  void ws() {
    while (p < end && isspace((unsigned char)*p)) ++p;
  }
  bool eat(char ch) {
    ws();
    if (p < end && *p == ch) {
      ++p;
      return true;
    }
    return false;
  }
  bool string(std::string* s) {
    ws();
    if (p >= end || *p != '"') return false;
    ++p;
    s->clear();
    while (p < end && *p != '"') {
      if (*p == '\\') return false;   // names and values here never need escapes
      s->push_back(*p++);
    }
    if (p >= end) return false;
    ++p;
    return true;
  }
  bool uint(uint64_t* v) {
    ws();
    if (p >= end || !isdigit((unsigned char)*p)) return false;
    uint64_t x = 0;
    while (p < end && isdigit((unsigned char)*p)) {
      x = x * 10 + (uint64_t)(*p - '0');
      if (x > 0xFFFFFFFFull) return false;
      ++p;
    }
    *v = x;
    return true;
  }
  // skip one value of any kind this format uses (string or unsigned integer)
  bool skip_scalar() {
    ws();
    std::string s;
    uint64_t v;
    if (p < end && *p == '"') return string(&s);
    return uint(&v);
  }
};

}  // namespace

bool tune_choice_valid(const dm_tune_choice& c) {
  if (c.reencode_warps > 16) return false;
  if (c.reencode_stages && (c.reencode_stages < 2 || c.reencode_stages > 4)) return false;
  if (c.reencode_obufs > 2) return false;
  if (c.x_staging > DM_STAGE_GLOBAL) return false;
  if (c.x8 > DM_X8_OFF) return false;
  return true;
}

dm_tune_key tune_key_of(const dm_column_in& in) {
  dm_tune_key k{};
  k.value_bytes = in.value_bytes;
  k.main_bits = in.main_bits;
  k.max_bits = bits_for(in.main_dict_len + in.delta_dict_len);
  k.log2_m = bit_length(in.main_dict_len);
  k.log2_d = bit_length(in.delta_dict_len);
  k.log2_main_rows = bit_length(in.main_rows);
  k.log2_delta_rows = bit_length(in.delta_rows);
  return k;
}

std::string tune_cache_to_json(const dm_tune_cache& c) {
  std::string s = "{\"format\": \"dmerge-tune-cache\", \"version\": 1, \"entries\": [";
  bool first = true;
  char buf[64];
  for (const auto& kv : c.entries) {
    dm_tune_key k{};
    k.value_bytes = std::get<0>(kv.first);
    k.main_bits = std::get<1>(kv.first);
    k.max_bits = std::get<2>(kv.first);
    k.log2_m = std::get<3>(kv.first);
    k.log2_d = std::get<4>(kv.first);
    k.log2_main_rows = std::get<5>(kv.first);
    k.log2_delta_rows = std::get<6>(kv.first);
    dm_tune_choice ch = kv.second;
    s += first ? "\n  {" : ",\n  {";
    first = false;
    for (size_t i = 0; i < kNumFields; ++i) {
      snprintf(buf, sizeof(buf), "%s\"%s\": %u", i ? ", " : "", kFields[i].name,
               *field_ptr(kFields[i], &k, &ch));
      s += buf;
    }
    s += "}";
  }
  s += "\n]}\n";
  return s;
}

bool tune_cache_from_json(const std::string& text, std::vector<std::pair<dm_tune_key, dm_tune_choice>>* out) {
  Reader r{text.data(), text.data() + text.size()};
  out->clear();
  if (!r.eat('{')) return false;
  bool seen_entries = false, seen_format = false;
  std::string name;
  if (!r.eat('}')) {
    do {
      if (!r.string(&name) || !r.eat(':')) return false;
      if (name == "entries") {
        seen_entries = true;
        if (!r.eat('[')) return false;
        if (r.eat(']')) continue;
        do {
          if (!r.eat('{')) return false;
          dm_tune_key k{};
          dm_tune_choice c{};
          bool seen[kNumFields] = {};
          if (!r.eat('}')) {
            do {
              std::string f;
              uint64_t v;
              if (!r.string(&f) || !r.eat(':') || !r.uint(&v)) return false;
              size_t i = 0;
              while (i < kNumFields && f != kFields[i].name) ++i;
              if (i == kNumFields) continue;   // a field of a later version: ignored
              if (seen[i]) return false;
              seen[i] = true;
              *field_ptr(kFields[i], &k, &c) = (uint32_t)v;
            } while (r.eat(','));
            if (!r.eat('}')) return false;
          }
          for (size_t i = 0; i < kNumFields; ++i)
            if (!seen[i]) return false;
          if (!tune_choice_valid(c)) return false;
          out->emplace_back(k, c);
        } while (r.eat(','));
        if (!r.eat(']')) return false;
      } else if (name == "format") {
        std::string v;
        if (!r.string(&v) || v != "dmerge-tune-cache") return false;
        seen_format = true;
      } else if (name == "version") {
        uint64_t v;
        if (!r.uint(&v) || v != 1) return false;
      } else if (!r.skip_scalar()) {
        return false;
      }
    } while (r.eat(','));
    if (!r.eat('}')) return false;
  }
  r.ws();
  return seen_entries && seen_format && r.p == r.end;
}

}  // namespace dm

extern "C" {

dm_status dm_tune_key_of(const dm_column_in* in, dm_tune_key* key) {
  if (!in || !key) return DM_EINVAL;
  *key = dm::tune_key_of(*in);
  return DM_OK;
}

dm_status dm_tune_cache_create(dm_tune_cache** out) {
  if (!out) return DM_EINVAL;
  *out = new (std::nothrow) dm_tune_cache();
  return *out ? DM_OK : DM_ENOMEM;
}

void dm_tune_cache_destroy(dm_tune_cache* c) { delete c; }

dm_status dm_tune_cache_put(dm_tune_cache* c, const dm_tune_key* key, const dm_tune_choice* choice) {
  if (!c || !key || !choice || !dm::tune_choice_valid(*choice)) return DM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  c->entries[dm_tune_cache::key_of(*key)] = *choice;
  c->size = c->entries.size();
  ++c->generation;
  return DM_OK;
}

dm_status dm_tune_cache_get(const dm_tune_cache* c, const dm_tune_key* key, dm_tune_choice* choice) {
  if (!c || !key || !choice) return DM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->entries.find(dm_tune_cache::key_of(*key));
  if (it == c->entries.end()) return DM_ENOENT;
  *choice = it->second;
  return DM_OK;
}

uint64_t dm_tune_cache_size(const dm_tune_cache* c) {
  if (!c) return 0;
  std::lock_guard<std::mutex> g(c->mu);
  return c->entries.size();
}

uint64_t dm_tune_cache_generation(const dm_tune_cache* c) {
  if (!c) return 0;
  std::lock_guard<std::mutex> g(c->mu);
  return c->generation;
}

dm_status dm_tune_cache_clear(dm_tune_cache* c) {
  if (!c) return DM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  c->entries.clear();
  c->size = 0;
  ++c->generation;
  return DM_OK;
}

dm_status dm_tune_cache_save(const dm_tune_cache* c, const char* path) {
  if (!c || !path) return DM_EINVAL;
  std::string text;
  {
    std::lock_guard<std::mutex> g(c->mu);
    text = dm::tune_cache_to_json(*c);
  }
  FILE* f = fopen(path, "wb");
  if (!f) return DM_EINVAL;
  const bool ok = fwrite(text.data(), 1, text.size(), f) == text.size();
  return (fclose(f) == 0 && ok) ? DM_OK : DM_EINVAL;
}

dm_status dm_tune_cache_load(dm_tune_cache* c, const char* path) {
  if (!c || !path) return DM_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return DM_ENOENT;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
  fclose(f);
  std::vector<std::pair<dm_tune_key, dm_tune_choice>> got;
  if (!dm::tune_cache_from_json(text, &got)) return DM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  for (const auto& e : got) c->entries[dm_tune_cache::key_of(e.first)] = e.second;
  c->size = c->entries.size();
  ++c->generation;
  return DM_OK;
}

}  // extern "C"
