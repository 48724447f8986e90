// Tuning table of the tcgen05 streaming passes (sketch, Gram-apply,
// projection, Gram of Alg. 3 steps 3, 4 and 10).
//
// A pass's launch shape has a few free parameters that do not change what
// it computes: the depth of its shared-memory ring, the CTAs per SM, the
// column width of a Gram stage (boxes of 64 columns) and the row height of a
// projection chunk.  The shape builders (stream_tc.cu) take them from fixed
// rules unless this table holds an entry for the pass's key
//   (pass, row bucket, MMA width N, n class),
// row bucket = the 16-rounded row count up to 128, then 256, 512, 1024 and
// "taller"; n class = 0 below 16,384 columns, 1 below 262,144, else 2.
// The table is filled by tt_tune_set / tt_tune_load (a text file written by
// the offline sweep paper_2308_01480_gb300/autotune.py).  Every entry is
// re-validated where it is applied; one that does not fit falls back to the
// fixed rules.  Workspace sizes do not depend on the table.
#include <mutex>
#include <map>
#include <cstdio>
#include <cstring>
#include <tuple>

#include "common.cuh"
#include "kernels.h"

namespace ttr {

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, TuneEntry> g_tune;

bool valid_entry(int op, const TuneEntry& e) {
  if (e.stages < 2 || e.stages > 8) return false;
  if (e.per_sm != 1 && e.per_sm != 2) return false;
  if (op == TT_PASS_GRAM) {
    if (e.kb != 1 && e.kb != 2 && e.kb != 4 && e.kb != 8) return false;
  } else if (e.kb != 0) {
    return false;
  }
  if (op == TT_PASS_PROJECT) {
    if (e.chunk_rows != 0 && e.chunk_rows != 64 && e.chunk_rows != 128) return false;
  } else if (e.chunk_rows != 0) {
    return false;
  }
  return true;
}

bool valid_key(int op, int rows, int npad, int nclass) {
  if (op < TT_PASS_SKETCH || op > TT_PASS_GRAM) return false;
  const bool short_rows = rows >= 16 && rows <= 128 && rows % 16 == 0;
  const bool tall_rows = rows == 256 || rows == 512 || rows == 1024 || rows == 4096;
  if (!short_rows && !tall_rows) return false;
  if (op == TT_PASS_GRAM && !short_rows) return false;
  if (npad < 16 || npad > 128 || npad % 16 != 0) return false;
  return nclass >= 0 && nclass <= 2;
}

}  // namespace

int tune_row_bucket(int64_t m) {
  if (m <= 128) return (int)((m + 15) / 16 * 16);
  if (m <= 256) return 256;
  if (m <= 512) return 512;
  if (m <= 1024) return 1024;
  return 4096;
}

int tune_n_class(int64_t n) { return n < 16384 ? 0 : (n < 262144 ? 1 : 2); }

bool tune_lookup(int op, int64_t m, int npad, int64_t n, TuneEntry* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune.empty()) return false;
  auto it = g_tune.find(std::make_tuple(op, tune_row_bucket(m), npad, tune_n_class(n)));
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

}  // namespace ttr

using ttr::TuneEntry;

extern "C" {

tt_status tt_tune_set(int op, int rows, int npad, int nclass, int stages, int per_sm, int kb, int chunk_rows) {
  if (!ttr::valid_key(op, rows, npad, nclass)) return TT_EINVAL;
  TuneEntry e{stages, per_sm, kb, chunk_rows};
  if (!ttr::valid_entry(op, e)) return TT_EINVAL;
  std::lock_guard<std::mutex> lk(ttr::g_tune_mu);
  ttr::g_tune[std::make_tuple(op, rows, npad, nclass)] = e;
  return TT_OK;
}

tt_status tt_tune_clear(void) {
  std::lock_guard<std::mutex> lk(ttr::g_tune_mu);
  ttr::g_tune.clear();
  return TT_OK;
}

int tt_tune_entries(void) {
  std::lock_guard<std::mutex> lk(ttr::g_tune_mu);
  return (int)ttr::g_tune.size();
}

tt_status tt_tune_get(int op, int rows, int npad, int nclass, int* out4) {
  if (!out4) return TT_EINVAL;
  std::lock_guard<std::mutex> lk(ttr::g_tune_mu);
  auto it = ttr::g_tune.find(std::make_tuple(op, rows, npad, nclass));
  if (it == ttr::g_tune.end()) return TT_EINVAL;
  out4[0] = it->second.stages;
  out4[1] = it->second.per_sm;
  out4[2] = it->second.kb;
  out4[3] = it->second.chunk_rows;
  return TT_OK;
}

// Text format: one entry per line, eight integers
//   op rows npad nclass stages per_sm kb chunk_rows
// anything after them on the line is ignored; lines starting with '#' and
// blank lines are skipped.  The whole file is checked before the table is
// replaced: on any bad line nothing changes and TT_EINVAL is returned.
tt_status tt_tune_load(const char* path) {
  if (!path) return TT_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return TT_EINVAL;
  std::map<std::tuple<int, int, int, int>, TuneEntry> next;
  char line[512];
  bool ok = true;
  while (std::fgets(line, sizeof line, f)) {
    const char* s = line;
    while (*s == ' ' || *s == '\t') ++s;
    if (*s == '#' || *s == '\n' || *s == '\r' || *s == '\0') continue;
    int v[8];
    if (std::sscanf(s, "%d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7]) != 8) {
      ok = false;
      break;
    }
    TuneEntry e{v[4], v[5], v[6], v[7]};
    if (!ttr::valid_key(v[0], v[1], v[2], v[3]) || !ttr::valid_entry(v[0], e)) {
      ok = false;
      break;
    }
    next[std::make_tuple(v[0], v[1], v[2], v[3])] = e;
  }
  std::fclose(f);
  if (!ok) return TT_EINVAL;
  std::lock_guard<std::mutex> lk(ttr::g_tune_mu);
  ttr::g_tune.swap(next);
  return TT_OK;
}

}  // extern "C"
