// Launch-shape tuner for the bit-sliced contribution kernel.
//
// For each shape class (value bits, lanes per row group, convention, and the
// base-2 logarithms of the row count and of the plane count) the first image
// of the class times a few launch shapes -- the row-group layout with warps
// per block (rows per block) and planes per tile (or equal plane spans per
// block), the warp-column layout with warps per block, then block-private
// shared-memory histograms against direct global atomics for the fastest
// shape -- on its own data, keeps the fastest, and reuses it for every later
// image of the class. With
// ecc_config.tuner_cache set, the table is read from and appended to that
// file (one JSON object per line).
#include "engine.h"

#include <cmath>
#include <cstdio>
#include <cstring>

namespace ecc {

int bits_nb(int dtype, int64_t bins);  // k_bits.cu

namespace {

int ilog2(int64_t v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

int lanes_per_row(int64_t nx) {
  int L = 1;
  while (L < (nx + 31) / 32 && L < 32) L <<= 1;
  return L;
}

}  // namespace

std::string Tuner::key(const LocalArgs& a) {
  char buf[96];
  snprintf(buf, sizeof buf, "nb%d_L%d_c%d_y%d_z%d", bits_nb(a.dtype, a.bins),
           lanes_per_row(a.n[2]), a.conv, ilog2(a.n[1]), ilog2(a.w_hi - a.w_lo));
  return buf;
}

void Tuner::load(const std::string& file) {
  path = file;
  FILE* f = std::fopen(file.c_str(), "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    char k[96] = {0};
    int w = 0, z = 0, hm = 0, lay = 0;
    float ms = 0;
    const int got = std::sscanf(
        line, " {\"key\": \"%95[^\"]\", \"warps\": %d, \"zc\": %d, \"ms\": %f, \"hist\": %d, \"layout\": %d",
        k, &w, &z, &ms, &hm, &lay);
    if (got >= 4 && w > 0 && z >= 0)
      table[k] = TuneChoice{w, z, ms, got >= 5 ? hm : 0, got >= 6 ? lay : 0};
  }
  std::fclose(f);
}

bool Tuner::lookup(const std::string& k, TuneChoice* c) {
  std::lock_guard<std::mutex> lk(mu);
  auto it = table.find(k);
  if (it == table.end()) return false;
  *c = it->second;
  return true;
}

void Tuner::store(const std::string& k, const TuneChoice& c) {
  std::lock_guard<std::mutex> lk(mu);
  table[k] = c;
  if (path.empty()) return;
  if (FILE* f = std::fopen(path.c_str(), "a")) {
    std::fprintf(f,
                 "{\"key\": \"%s\", \"warps\": %d, \"zc\": %d, \"ms\": %.6f, \"hist\": %d, "
                 "\"layout\": %d}\n",
                 k.c_str(), c.warps, c.zc, c.ms, c.hist, c.layout);
    std::fclose(f);
  }
}

// Times the candidate shapes on this launch (its data and stream); the
// VCEC accumulator is left dirty, the caller clears it afterwards.
int tune_bits(ecc_handle* h, const LocalArgs& base, TuneChoice* best) {
  const int L = lanes_per_row(base.n[2]);
  const int R = 32 / L;
  const int64_t planes = base.w_hi - base.w_lo;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
    if (e0) cudaEventDestroy(e0);
    return cuda_err(h, e, "tuner");
  }
  best->ms = 1e30f;
  best->warps = 0;
  best->zc = 0;
  int rc = ECC_OK;
  // one warm launch, then one timed launch of a candidate
  auto time_one = [&](const LocalArgs& a, float* ms) -> int {
    int64_t cnt = 0;
    if ((e = launch_local(a, h->num_sms, &cnt)) || (e = cudaEventRecord(e0, a.stream)) ||
        (e = launch_local(a, h->num_sms, &cnt)) || (e = cudaEventRecord(e1, a.stream)))
      return cuda_err(h, e, "tuner launch");
    h->launches += cnt;
    int r = wait_event(h, e1, 300LL * 1000 * 1000);
    if (r) return r;
    if ((e = cudaEventElapsedTime(ms, e0, e1))) return cuda_err(h, e, "tuner timing");
    return ECC_OK;
  };
  // row groups: warps per block x planes per tile
  for (int W : {4, 8, 16}) {
    if (W * R < 3 || W * R > 512) continue;
    for (int zc : {0, 16, 32, 64, 128}) {  // 0: balanced spans
      if (zc > 2 * planes && zc != 16) continue;
      LocalArgs a = base;
      a.layout = 1;
      a.warps = W;
      a.zc = zc;
      a.hist = 0;
      float ms = 0;
      if ((rc = time_one(a, &ms))) break;
      if (ms < best->ms) *best = TuneChoice{W, zc, ms, 0, 1};
    }
    if (rc) break;
  }
  // warp columns: warps per block
  for (int W : {4, 8}) {
    if (rc) break;
    LocalArgs a = base;
    a.layout = 2;
    a.warps = W;
    a.zc = 0;
    a.hist = 0;
    float ms = 0;
    if ((rc = time_one(a, &ms))) break;
    if (ms < best->ms) *best = TuneChoice{W, 0, ms, 0, 2};
  }
  // histogram privatisation for the fastest shape: shared memory or global
  if (!rc && best->warps > 0 && base.bins <= kSmemBinsMax) {
    LocalArgs a = base;
    a.layout = best->layout;
    a.warps = best->warps;
    a.zc = best->zc;
    a.hist = 2;
    float ms = 0;
    if (!(rc = time_one(a, &ms)) && ms < best->ms)
      *best = TuneChoice{best->warps, best->zc, ms, 2, best->layout};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace ecc
