// TEST INFRASTRUCTURE — CPU oracle of the per-column delta-to-main merge.
//
// A plain, single-threaded, deliberately unoptimised statement of what one
// column merge computes (Krueger et al., "Fast Updates on Read-Optimized
// Databases Using Multi-Core CPUs", Section 5).  Only the tests, the smoke
// check and the benchmark's CPU-baseline leg load it; the product path never
// does.  It shares no source with the CUDA library.
//
// Data conventions (the paper fixes none of these; they are the readings the
// library documents as well):
//   * keys are unsigned integers of w = 4, 8 or 16 bytes; a 16-byte key is
//     the pair {uint64 hi, uint64 lo} compared hi first;
//   * a packed code vector stores code i in stream bits [i*b, (i+1)*b),
//     least significant bit first, stream bit k being bit k%32 of 32-bit
//     word k/32, padded with zero bits to a whole number of 16-byte units;
//   * the delta partition is an insertion-order dictionary D_dict (distinct
//     values, duplicates tolerated) plus uint32 row codes into it, so X_D is
//     indexed by insertion code.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

namespace {

enum {
  ORACLE_OK = 0,
  ORACLE_BAD_ARG = 1,   // widths, sizes or missing buffers
  ORACLE_UNSORTED = 2,  // U_M not strictly increasing
  ORACLE_BAD_CODE = 3,  // a main code >= |U_M| or a delta code >= |D_dict|
};

// A key widened to (hi, lo): w = 4 and w = 8 keys have hi = 0.
struct Key {
  uint64_t hi, lo;
};

bool operator<(const Key& a, const Key& b) { return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo; }
bool operator==(const Key& a, const Key& b) { return a.hi == b.hi && a.lo == b.lo; }

Key load_key(const void* base, uint64_t i, uint32_t w) {
  const unsigned char* p = static_cast<const unsigned char*>(base) + i * w;
  Key k{0, 0};
  if (w == 4) {
    uint32_t v;
    std::memcpy(&v, p, 4);
    k.lo = v;
  } else if (w == 8) {
    std::memcpy(&k.lo, p, 8);
  } else {
    std::memcpy(&k.hi, p, 8);
    std::memcpy(&k.lo, p + 8, 8);
  }
  return k;
}

void store_key(void* base, uint64_t i, uint32_t w, const Key& k) {
  unsigned char* p = static_cast<unsigned char*>(base) + i * w;
  if (w == 4) {
    uint32_t v = static_cast<uint32_t>(k.lo);
    std::memcpy(p, &v, 4);
  } else if (w == 8) {
    std::memcpy(p, &k.lo, 8);
  } else {
    std::memcpy(p, &k.hi, 8);
    std::memcpy(p + 8, &k.lo, 8);
  }
}

bool width_ok(uint32_t w) { return w == 4 || w == 8 || w == 16; }

// Number of 32-bit words of a stream of n codes at b bits.
uint64_t words_for(uint64_t n, uint32_t b) { return ((n * b + 127) / 128) * 4; }

// Code i of an LSB-first stream at b bits.
uint32_t unpack_code(const uint32_t* words, uint64_t nwords, uint64_t i, uint32_t b) {
  if (b == 0) return 0;
  uint64_t bit = i * b;
  uint64_t k = bit / 32;
  uint64_t window = words[k];
  if (k + 1 < nwords) window |= static_cast<uint64_t>(words[k + 1]) << 32;
  uint64_t mask = (b == 32) ? 0xFFFFFFFFull : ((1ull << b) - 1);
  return static_cast<uint32_t>((window >> (bit % 32)) & mask);
}

// OR code v into position i of an LSB-first stream at b bits.
void pack_code(uint32_t* words, uint64_t i, uint32_t b, uint32_t v) {
  if (b == 0) return;
  uint64_t bit = i * b;
  uint64_t k = bit / 32;
  uint32_t sh = static_cast<uint32_t>(bit % 32);
  uint64_t shifted = static_cast<uint64_t>(v) << sh;
  words[k] |= static_cast<uint32_t>(shifted);
  if (sh + b > 32) words[k + 1] |= static_cast<uint32_t>(shifted >> 32);
}

}  // namespace

extern "C" {

// Words of a packed stream of n codes at b bits (16-byte padded).
uint64_t oracle_packed_words(uint64_t n, uint32_t b) { return words_for(n, b); }

// Step 2(a), Eq. 4: E'_C = ceil(log2 u); 0 when u <= 1 (the paper is silent
// there; zero bits is the least width that still decodes every code, 0).
uint32_t oracle_new_width(uint64_t u) {
  uint32_t b = 0;
  while (b < 64 && (1ull << b) < u) ++b;
  return b;
}

// Step 1(a), Section 5.1 with the tuple-id map of Section 5.3: the sorted
// delta dictionary U_D together with perm[j] = insertion code of U_D[j].
// Equal values (duplicates in D_dict) stay in insertion order.
int oracle_sort_delta(uint32_t w, const void* delta_dict, uint64_t d, void* ud_out, uint32_t* perm) {
  if (!width_ok(w)) return ORACLE_BAD_ARG;
  std::vector<std::pair<Key, uint64_t>> pairs(d);
  for (uint64_t k = 0; k < d; ++k) pairs[k] = {load_key(delta_dict, k, w), k};
  std::sort(pairs.begin(), pairs.end(), [](const auto& a, const auto& b) {
    if (a.first == b.first) return a.second < b.second;
    return a.first < b.first;
  });
  for (uint64_t j = 0; j < d; ++j) {
    store_key(ud_out, j, w, pairs[j].first);
    perm[j] = static_cast<uint32_t>(pairs[j].second);
  }
  return ORACLE_OK;
}

// Step 1(b), Section 5.1, with the translation tables of Section 5.3: one
// pass over U_M and U_D with an iterator on each.  The smaller current value
// is appended to U' and its output index is recorded in X_M (main) or X_D
// (delta, at the value's insertion code perm[j]); on equal values the value
// is appended once, both tables receive the same index and both iterators
// advance.  A delta value equal to the value appended last (a duplicate
// inside D_dict) takes that value's index and appends nothing.
int oracle_merge_dicts(uint32_t w, const void* um, uint64_t m, const void* ud, const uint32_t* perm,
                       uint64_t d, void* unew, uint32_t* xm, uint32_t* xd, uint64_t* u_out) {
  if (!width_ok(w)) return ORACLE_BAD_ARG;
  uint64_t i = 0, j = 0, u = 0;
  Key last{0, 0};
  auto append = [&](const Key& v) {
    store_key(unew, u, w, v);
    last = v;
    return static_cast<uint32_t>(u++);
  };
  while (i < m && j < d) {
    Key a = load_key(um, i, w);
    Key b = load_key(ud, j, w);
    if (u > 0 && b == last) {
      xd[perm[j]] = static_cast<uint32_t>(u - 1);
      ++j;
    } else if (a < b) {
      xm[i] = append(a);
      ++i;
    } else if (b < a) {
      xd[perm[j]] = append(b);
      ++j;
    } else {
      uint32_t c = append(a);
      xm[i] = c;
      xd[perm[j]] = c;
      ++i;
      ++j;
    }
  }
  while (i < m) {
    xm[i] = append(load_key(um, i, w));
    ++i;
  }
  while (j < d) {
    Key b = load_key(ud, j, w);
    if (u > 0 && b == last)
      xd[perm[j]] = static_cast<uint32_t>(u - 1);
    else
      xd[perm[j]] = append(b);
    ++j;
  }
  *u_out = u;
  return ORACLE_OK;
}

// Step 2(b), Section 5.3 and Eq. 11: new main code i = X_M[M[i]], then the
// delta rows r get X_D[D[r]], all written at width b_new into a zeroed
// stream of N_M + N_D codes.
int oracle_reencode(const uint32_t* main_words, uint32_t b, uint64_t n_main, const uint32_t* dcodes,
                    uint64_t n_delta, const uint32_t* xm, uint64_t m, const uint32_t* xd, uint64_t d,
                    uint32_t b_new, uint32_t* out_words) {
  if (b > 32 || b_new > 32) return ORACLE_BAD_ARG;
  uint64_t n_out = n_main + n_delta;
  uint64_t in_words = words_for(n_main, b);
  std::memset(out_words, 0, words_for(n_out, b_new) * 4);
  for (uint64_t i = 0; i < n_main; ++i) {
    uint32_t c = unpack_code(main_words, in_words, i, b);
    if (c >= m) return ORACLE_BAD_CODE;
    pack_code(out_words, i, b_new, xm[c]);
  }
  for (uint64_t r = 0; r < n_delta; ++r) {
    uint32_t c = dcodes[r];
    if (c >= d) return ORACLE_BAD_CODE;
    pack_code(out_words, n_main + r, b_new, xd[c]);
  }
  return ORACLE_OK;
}

// Input checks: widths, U_M strictly increasing, every code in range, and
// u <= 2^32 so that new codes fit uint32.
int oracle_validate(uint32_t w, const void* um, uint64_t m, const uint32_t* main_words, uint32_t b,
                    uint64_t n_main, uint64_t d, const uint32_t* dcodes, uint64_t n_delta) {
  if (!width_ok(w) || b > 32) return ORACLE_BAD_ARG;
  if (m + d > (1ull << 32)) return ORACLE_BAD_ARG;
  if (b < oracle_new_width(m)) return ORACLE_BAD_ARG;
  if ((n_main > 0 && m == 0) || (n_delta > 0 && d == 0)) return ORACLE_BAD_ARG;
  for (uint64_t i = 1; i < m; ++i)
    if (!(load_key(um, i - 1, w) < load_key(um, i, w))) return ORACLE_UNSORTED;
  uint64_t in_words = words_for(n_main, b);
  for (uint64_t i = 0; i < n_main; ++i)
    if (unpack_code(main_words, in_words, i, b) >= m) return ORACLE_BAD_CODE;
  for (uint64_t r = 0; r < n_delta; ++r)
    if (dcodes[r] >= d) return ORACLE_BAD_CODE;
  return ORACLE_OK;
}

// The whole column merge (Section 5, Steps 1 and 2 with the Section 5.3
// modifications).  Caller-owned outputs: unew holds m + d keys, xm m
// entries, xd d entries, out_words oracle_packed_words(n_main + n_delta,
// oracle_new_width(m + d)) words.
int oracle_merge_column(uint32_t w, const void* um, uint64_t m, const uint32_t* main_words, uint32_t b,
                        uint64_t n_main, const void* ddict, uint64_t d, const uint32_t* dcodes,
                        uint64_t n_delta, void* unew, uint32_t* xm, uint32_t* xd, uint32_t* out_words,
                        uint64_t* u_out, uint32_t* b_new_out) {
  int rc = oracle_validate(w, um, m, main_words, b, n_main, d, dcodes, n_delta);
  if (rc != ORACLE_OK) return rc;
  std::vector<unsigned char> ud(d * w + 1);
  std::vector<uint32_t> perm(d + 1);
  rc = oracle_sort_delta(w, ddict, d, ud.data(), perm.data());
  if (rc != ORACLE_OK) return rc;
  rc = oracle_merge_dicts(w, um, m, ud.data(), perm.data(), d, unew, xm, xd, u_out);
  if (rc != ORACLE_OK) return rc;
  *b_new_out = oracle_new_width(*u_out);
  return oracle_reencode(main_words, b, n_main, dcodes, n_delta, xm, m, xd, d, *b_new_out, out_words);
}

// Step 2(b) by the unmodified route of Section 5.2 (Eq. 5): decode each
// main code through U_M, then binary-search the value in U'; delta rows
// search their value directly.  Same output as the translation-table route.
int oracle_naive_reencode(uint32_t w, const void* um, uint64_t m, const uint32_t* main_words, uint32_t b,
                          uint64_t n_main, const void* ddict, uint64_t d, const uint32_t* dcodes,
                          uint64_t n_delta, const void* unew, uint64_t u, uint32_t b_new,
                          uint32_t* out_words) {
  if (!width_ok(w) || b > 32 || b_new > 32) return ORACLE_BAD_ARG;
  std::vector<Key> dict(u);
  for (uint64_t k = 0; k < u; ++k) dict[k] = load_key(unew, k, w);
  uint64_t n_out = n_main + n_delta;
  uint64_t in_words = words_for(n_main, b);
  std::memset(out_words, 0, words_for(n_out, b_new) * 4);
  auto find = [&](const Key& v, uint32_t* code) {
    auto it = std::lower_bound(dict.begin(), dict.end(), v);
    if (it == dict.end() || !(*it == v)) return false;
    *code = static_cast<uint32_t>(it - dict.begin());
    return true;
  };
  for (uint64_t i = 0; i < n_main; ++i) {
    uint32_t c = unpack_code(main_words, in_words, i, b), code;
    if (c >= m || !find(load_key(um, c, w), &code)) return ORACLE_BAD_CODE;
    pack_code(out_words, i, b_new, code);
  }
  for (uint64_t r = 0; r < n_delta; ++r) {
    uint32_t c = dcodes[r], code;
    if (c >= d || !find(load_key(ddict, c, w), &code)) return ORACLE_BAD_CODE;
    pack_code(out_words, n_main + r, b_new, code);
  }
  return ORACLE_OK;
}

// Delta ingest (Section 4, Figure 5): values appended to the delta
// partition in arrival order.  The partition's dictionary holds each
// distinct value once; here it lists them in order of first arrival, and
// each tuple's code is the position of its value in that list (the first
// arrival of a value takes the next code, later arrivals reuse it).
int oracle_ingest_delta(uint32_t w, const void* values, uint64_t n, void* dict_out, uint32_t* codes,
                        uint64_t* d_out) {
  if (!width_ok(w) || (n && (!values || !dict_out || !codes)) || !d_out) return ORACLE_BAD_ARG;
  std::map<Key, uint32_t> seen;
  uint64_t d = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const Key k = load_key(values, i, w);
    auto it = seen.find(k);
    if (it == seen.end()) {
      seen.emplace(k, static_cast<uint32_t>(d));
      store_key(dict_out, d, w, k);
      codes[i] = static_cast<uint32_t>(d);
      ++d;
    } else {
      codes[i] = it->second;
    }
  }
  *d_out = d;
  return ORACLE_OK;
}

}  // extern "C"
