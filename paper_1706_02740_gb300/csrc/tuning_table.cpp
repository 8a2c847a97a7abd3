// Tuned launch geometries kept across batches and processes.  The autotuner's choice depends on
// the shapes of a batch's transforms (N and s set the nodes, the primes and the chirp lengths),
// the window and the precision, so the table is keyed by the class floor(log2 N), floor(log2 s),
// kappa, precision of a batch whose plans all share it: sft_batch_autotune stores its choice
// there, and sft_batch_create starts such a batch from the stored entry.  The file form is text,
// one entry per line after a header line: 17 integers, the four key fields, then
// resample_threads, resample_regcap, bin_threads, dft_per_cta[0..8], dft_two_ctas.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "guard.h"
#include "sft_internal.h"
#include "tuning_table.h"

namespace sft {

namespace {

constexpr const char* kHeader = "# sft tuning table v1";

using KeyTuple = std::tuple<int32_t, int32_t, int32_t, int32_t>;

struct Table {
  std::mutex mu;
  std::map<KeyTuple, sft_tuning> entries;
};

Table& table() {
  static Table t;
  return t;
}

KeyTuple as_tuple(const TuneKey& k) { return KeyTuple(k.log2n, k.log2s, k.kappa, k.prec); }

int32_t floor_log2(int64_t x) {
  int32_t r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

bool key_valid(int64_t N, int32_t s, int32_t kappa, int32_t prec, std::string* why) {
  if (N < 2 || s < 1 || kappa < 1 || kappa > kMaxKappa || (prec != SFT_FP32 && prec != SFT_FP64)) {
    *why = "need N >= 2, s >= 1, 1 <= kappa <= " + std::to_string(kMaxKappa) + ", precision 0 or 1";
    return false;
  }
  return true;
}

}  // namespace

TuneKey tune_key(int64_t N, int32_t s, int32_t kappa, int32_t prec) {
  return TuneKey{floor_log2(N), floor_log2(s), kappa, prec};
}

bool same_key(const TuneKey& a, const TuneKey& b) { return as_tuple(a) == as_tuple(b); }

bool tuning_table_find(const TuneKey& k, sft_tuning* out) {
  Table& T = table();
  std::lock_guard<std::mutex> g(T.mu);
  const auto it = T.entries.find(as_tuple(k));
  if (it == T.entries.end()) return false;
  *out = it->second;
  return true;
}

void tuning_table_store(const TuneKey& k, const sft_tuning& t) {
  Table& T = table();
  std::lock_guard<std::mutex> g(T.mu);
  T.entries[as_tuple(k)] = t;
}

}  // namespace sft

extern "C" {

sft_status sft_tuning_table_put(int64_t N, int32_t s, int32_t kappa, int32_t precision,
                                const sft_tuning* t) {
  return sft::guarded("sft_tuning_table_put", [&]() -> sft_status {
    using namespace sft;
    std::string why;
    if (!t) { set_error("sft_tuning_table_put: NULL tuning"); return SFT_EINVAL; }
    if (!key_valid(N, s, kappa, precision, &why) || !tuning_valid(*t, &why)) {
      set_error("sft_tuning_table_put: " + why);
      return SFT_EINVAL;
    }
    tuning_table_store(tune_key(N, s, kappa, precision), *t);
    return SFT_OK;
  });
}

sft_status sft_tuning_table_get(int64_t N, int32_t s, int32_t kappa, int32_t precision,
                                sft_tuning* t) {
  using namespace sft;
  std::string why;
  if (!t) { set_error("sft_tuning_table_get: NULL tuning"); return SFT_EINVAL; }
  if (!key_valid(N, s, kappa, precision, &why)) {
    set_error("sft_tuning_table_get: " + why);
    return SFT_EINVAL;
  }
  if (!tuning_table_find(tune_key(N, s, kappa, precision), t)) {
    set_error("sft_tuning_table_get: no entry for this class");
    return SFT_EINVAL;
  }
  return SFT_OK;
}

int32_t sft_tuning_table_size(void) {
  sft::Table& T = sft::table();
  std::lock_guard<std::mutex> g(T.mu);
  return (int32_t)T.entries.size();
}

void sft_tuning_table_clear(void) {
  sft::Table& T = sft::table();
  std::lock_guard<std::mutex> g(T.mu);
  T.entries.clear();
}

sft_status sft_tuning_table_save(const char* path) {
  return sft::guarded("sft_tuning_table_save", [&]() -> sft_status {
    using namespace sft;
    if (!path) { set_error("sft_tuning_table_save: NULL path"); return SFT_EINVAL; }
    std::vector<std::pair<KeyTuple, sft_tuning>> rows;
    {
      Table& T = table();
      std::lock_guard<std::mutex> g(T.mu);
      rows.assign(T.entries.begin(), T.entries.end());
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) { set_error(std::string("sft_tuning_table_save: cannot write ") + tmp); return SFT_EINVAL; }
    bool ok = fprintf(f, "%s\n", kHeader) > 0;
    for (const auto& r : rows) {
      const sft_tuning& t = r.second;
      ok = ok && fprintf(f, "%d %d %d %d %d %d %d", std::get<0>(r.first), std::get<1>(r.first),
                         std::get<2>(r.first), std::get<3>(r.first), t.resample_threads,
                         t.resample_regcap, t.bin_threads) > 0;
      for (int c = 0; c < 9; ++c) ok = ok && fprintf(f, " %d", t.dft_per_cta[c]) > 0;
      ok = ok && fprintf(f, " %d\n", t.dft_two_ctas) > 0;
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
      remove(tmp.c_str());
      set_error(std::string("sft_tuning_table_save: write failed: ") + path);
      return SFT_EINVAL;
    }
    return SFT_OK;
  });
}

sft_status sft_tuning_table_load(const char* path) {
  return sft::guarded("sft_tuning_table_load", [&]() -> sft_status {
    using namespace sft;
    if (!path) { set_error("sft_tuning_table_load: NULL path"); return SFT_EINVAL; }
    FILE* f = fopen(path, "r");
    if (!f) { set_error(std::string("sft_tuning_table_load: cannot read ") + path); return SFT_EINVAL; }
    std::vector<std::pair<KeyTuple, sft_tuning>> rows;
    char line[512];
    int lineno = 0;
    std::string err;
    while (err.empty() && fgets(line, sizeof(line), f)) {
      ++lineno;
      if (lineno == 1) {
        if (strncmp(line, kHeader, strlen(kHeader)) != 0) err = "not a tuning table (header)";
        continue;
      }
      if (line[0] == '\n' || line[0] == '\0') continue;
      int v[17];
      char extra;
      const int got = sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %c", &v[0],
                             &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7], &v[8], &v[9], &v[10],
                             &v[11], &v[12], &v[13], &v[14], &v[15], &v[16], &extra);
      if (got != 17) {
        err = "line " + std::to_string(lineno) + ": expected 17 integers";
        break;
      }
      sft_tuning t;
      t.resample_threads = v[4];
      t.resample_regcap = v[5];
      t.bin_threads = v[6];
      for (int c = 0; c < 9; ++c) t.dft_per_cta[c] = v[7 + c];
      t.dft_two_ctas = v[16];
      std::string why;
      const bool key_ok = v[0] >= 1 && v[0] <= 62 && v[1] >= 0 && v[1] <= 31 && v[2] >= 1 &&
                          v[2] <= kMaxKappa && (v[3] == SFT_FP32 || v[3] == SFT_FP64);
      if (!key_ok) err = "line " + std::to_string(lineno) + ": bad key";
      else if (!tuning_valid(t, &why)) err = "line " + std::to_string(lineno) + ": " + why;
      else rows.push_back({KeyTuple(v[0], v[1], v[2], v[3]), t});
    }
    if (err.empty() && lineno == 0) err = "empty file";
    fclose(f);
    if (!err.empty()) {
      set_error("sft_tuning_table_load: " + err + " (nothing merged)");
      return SFT_EINVAL;
    }
    Table& T = table();
    std::lock_guard<std::mutex> g(T.mu);
    for (const auto& r : rows) T.entries[r.first] = r.second;
    return SFT_OK;
  });
}

}  // extern "C"
