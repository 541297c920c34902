// sp_tune.cu -- the autotuner: leaf size, recompression chunk shape and the
// small-problem GEMM tiling chosen by timing whole projectors.
//
// Not part of the paper (its experiments fix n_min = 250 for tridiagonal and
// 500 for banded matrices, Sec. 6, and study the time as a function of n_min
// in the tridiagonal example of Sec. 6.2).  Here the choice is measured on the
// GPU: the projector of a tuning problem (the leading min(n, 16384) block of
// the caller's band, same shift) is timed for every candidate leaf size in
// {64, 128, 256, 512} (at least 2b, at most half the tuning order), then, at
// the best leaf, for TSQR chunks of 256, 512 and 1024 rows and with the 16 x 16
// small-problem GEMM tiles on and off (coordinate descent).  Results are kept
// in a cache file of JSON lines keyed by (floor(log2 n), b, precision), read
// back by sp_ctx_load_tuning; a leaf argument of 0 then takes the tuned leaf.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>

#include "sp_internal.h"

namespace sp {
namespace {

int nbucket(int64_t n) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= n) ++l;
  return l;
}

// one cache line: {"nbucket": 16, "b": 1, "precision": 0, "leaf": 256, ...}
bool parse_line(const std::string& line, sp_ctx::TunedLeaf& e, double* ms) {
  auto field = [&](const char* key, double* out) {
    const std::string k = std::string("\"") + key + "\"";
    const size_t p = line.find(k);
    if (p == std::string::npos) return false;
    const size_t c = line.find(':', p + k.size());
    if (c == std::string::npos) return false;
    *out = std::strtod(line.c_str() + c + 1, nullptr);
    return true;
  };
  double v[7];
  const char* keys[7] = {"nbucket", "b", "precision", "leaf", "tsqr_chunk", "small_tiles", "ms"};
  for (int i = 0; i < 7; ++i)
    if (!field(keys[i], &v[i])) return false;
  e = sp_ctx::TunedLeaf{(int)v[0], (int)v[1], (int)v[2], (int)v[3], (int)v[4], (int)v[5]};
  if (ms) *ms = v[6];
  return e.leaf > 0 && e.tsqr_chunk > 0;
}

std::vector<std::pair<sp_ctx::TunedLeaf, double>> read_cache(const char* path) {
  std::vector<std::pair<sp_ctx::TunedLeaf, double>> out;
  if (!path || !*path) return out;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    sp_ctx::TunedLeaf e;
    double ms = 0.0;
    if (parse_line(line, e, &ms)) out.push_back({e, ms});
  }
  return out;
}

}  // namespace

// Leaf from the context's tuning table for (n, b), else the rule 64 / 128 /
// 256 by n (at least 2b).  Also applies the entry's chunk and tile policy.
int tuned_leaf(sp_ctx* ctx, int64_t n, int b) {
  const int nb = nbucket(n);
  const sp_ctx::TunedLeaf* best = nullptr;
  for (const auto& e : ctx->tuned)
    if (e.b == b && (!best || std::abs(e.nbucket - nb) < std::abs(best->nbucket - nb))) best = &e;
  if (best && std::abs(best->nbucket - nb) <= 1) return std::max(best->leaf, std::max(2 * b, 2));
  const int leaf = n <= 2048 ? 64 : (n <= 8192 ? 128 : 256);
  return std::max(leaf, std::max(2 * b, 2));
}

}  // namespace sp

using namespace sp;

extern "C" {

int sp_ctx_set_tuning(sp_ctx_t ctx, int32_t tsqr_chunk, int32_t small_tiles) {
  if (!ctx || tsqr_chunk < 32 || tsqr_chunk > 8192) return SP_EINVAL;
  ctx->tsqr_chunk = tsqr_chunk;
  ctx->small_tiles = small_tiles != 0;
  return SP_OK;
}

int sp_ctx_load_tuning(sp_ctx_t ctx, const char* cache_path) {
  if (!ctx || !cache_path) return SP_EINVAL;
  ctx->tuned.clear();
  for (const auto& e : read_cache(cache_path)) ctx->tuned.push_back(e.first);
  return SP_OK;
}

int sp_autotune(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu, double tol,
                int32_t precision, const char* cache_path, sp_tune_result* out) {
  if (!ctx || !ab || !out || n < 2 || b < 1 || ldab < b + 1 || !(tol > 0.0)) return SP_EINVAL;
  std::memset(out, 0, sizeof(*out));
  const int nb = nbucket(n);
  for (const auto& e : read_cache(cache_path))
    if (e.first.nbucket == nb && e.first.b == b && e.first.precision == precision) {
      out->leaf = e.first.leaf;
      out->tsqr_chunk = e.first.tsqr_chunk;
      out->small_tiles = e.first.small_tiles;
      out->ms = e.second;
      out->trials = 0;
      out->n_tuned = 0;
      ctx->tuned.push_back(e.first);
      return SP_OK;
    }
  const int64_t nt = std::min<int64_t>(n, 16384);
  const int saved_chunk = ctx->tsqr_chunk;
  const bool saved_tiles = ctx->small_tiles;
  sp_qdwh_opts o;
  sp_qdwh_opts_default(&o);
  o.precision = precision;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SP_ECUDA;
  int trials = 0;
  // time of one projector of the tuning problem, or a negative status
  auto run = [&](int leaf, int chunk, bool tiles, double* ms) -> int {
    ctx->tsqr_chunk = chunk;
    ctx->small_tiles = tiles;
    cudaEventRecord(e0, ctx->stream);
    sp_hodlr_t A = nullptr, S = nullptr, P = nullptr;
    int rc = sp_hodlr_from_band(ctx, nt, b, ab, ldab, mu, leaf, tol, 0, &A);
    if (rc == SP_OK) rc = sp_qdwh_sign(ctx, A, &o, &S, nullptr);
    if (rc == SP_OK) rc = sp_projector(ctx, S, &P);
    double tr = 0.0;
    if (rc == SP_OK) rc = sp_trace(ctx, P, &tr);
    sp_hodlr_destroy(A);
    sp_hodlr_destroy(S);
    sp_hodlr_destroy(P);
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t;
    ++trials;
    return rc;
  };
  double ms = 0.0;
  int rc = run(std::max(64, 2 * b), 512, true, &ms);  // warm-up (first-touch allocations)
  std::vector<int> leaves;
  for (int leaf : {64, 128, 256, 512})
    if (leaf >= 2 * b && leaf <= std::max<int64_t>(nt / 2, 2 * b)) leaves.push_back(leaf);
  int best_leaf = leaves.empty() ? 2 * b : leaves[0];
  double best = 1e300;
  for (int leaf : leaves) {
    const int r = run(leaf, 512, true, &ms);
    if (r != SP_OK) {
      rc = r;
      continue;
    }
    rc = SP_OK;
    if (ms < best) {
      best = ms;
      best_leaf = leaf;
    }
  }
  int best_chunk = 512;
  bool best_tiles = true;
  if (best < 1e300) {
    for (int chunk : {256, 1024})
      if (run(best_leaf, chunk, true, &ms) == SP_OK && ms < best) {
        best = ms;
        best_chunk = chunk;
      }
    if (run(best_leaf, best_chunk, false, &ms) == SP_OK && ms < best) {
      best = ms;
      best_tiles = false;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tsqr_chunk = saved_chunk;
  ctx->small_tiles = saved_tiles;
  if (!(best < 1e300)) {
    if (ctx->err.empty()) ctx->err = "sp_autotune: no candidate ran";
    return rc != SP_OK ? rc : SP_EINTERNAL;
  }
  out->leaf = best_leaf;
  out->tsqr_chunk = best_chunk;
  out->small_tiles = best_tiles ? 1 : 0;
  out->ms = best;
  out->trials = trials;
  out->n_tuned = nt;
  const sp_ctx::TunedLeaf e{nb, b, precision, best_leaf, best_chunk, best_tiles ? 1 : 0};
  ctx->tuned.push_back(e);
  if (cache_path && *cache_path) {
    std::ofstream f(cache_path, std::ios::app);
    if (!f) {
      ctx->err = std::string("sp_autotune: cannot append to ") + cache_path;
      return SP_EINVAL;
    }
    f << "{\"nbucket\": " << nb << ", \"b\": " << b << ", \"precision\": " << precision << ", \"leaf\": " << best_leaf
      << ", \"tsqr_chunk\": " << best_chunk << ", \"small_tiles\": " << (best_tiles ? 1 : 0) << ", \"ms\": " << best
      << ", \"n_tuned\": " << nt << "}\n";
  }
  return SP_OK;
}

}  // extern "C"
