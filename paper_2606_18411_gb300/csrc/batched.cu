// Batched MRCQR (many independent factorizations of uneven m and n: the
// repeated QRs of block Krylov and randomized-SVD power steps, Sec. II-C):
// one workspace for the whole batch, and per phase one grouped launch over a
// work list of {problem, block} items (plus one per kernel variant), so
// small problems share the GPU instead of launching dozens of kernels each.
// The precision ladder of every problem (Sec. II-C) runs level by level:
// items of level L skip themselves unless their problem is active at L.
//
// With emulated FP64 products (the default, as in mrcqr_factor) the heavy
// phases -- the FP64 sketch, W = A R_s^{-1}, the Gram, Q = W R_c^{-1} and the
// check -- run as grouped persistent tensor-core kernels too: one launch per
// kernel walks the {problem, row block / tile} items of every problem
// (oz_per_problem = 1 instead runs the single-problem kernels per problem on
// side streams).  fp64_products = 1 runs every phase grouped with FP64 FMA
// kernels.
//
// A plan (mrcqr_batched_plan_*) keeps the workspace, the uploaded work lists
// and optionally the whole launch sequence captured as a CUDA graph, so a
// repeated batch replays with one graph launch.  The tuner picks the SYRK
// split size and the sketch chunk size by timing the grouped kernels on the
// batch itself; results are cached per batch shape (and in the file named by
// MRCQR_TUNE_CACHE, if set).
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/mrcqr.h"
#include "kernels.h"

using namespace mrcqr;

namespace {

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

enum Kind {
  K_INIT, K_SAMPLE, K_COSTAB, K_SKETCH, K_SKREDUCE, K_SQR, K_TRSM, K_SYRK, K_GREDUCE, K_CHOL, K_TRINV, K_RMUL,
  K_FINALIZE, K_CHECK, K_EREDUCE, K_JUDGE, K_PUBLISH,
  // emulated-FP64 phases of one problem (param = problem) between a fork and a join of the side streams
  K_FORK, K_JOIN, K_OZ_SKETCH, K_OZ_STAGE2A, K_OZ_STAGE2B,
  // grouped emulated-FP64 kernels (param = 1: the check's Gram)
  KG_OZ_COLHI, KG_OZ_SKETCH, KG_OZ_SKREDUCE, KG_OZ_ROWSCALE, KG_OZ_PREPR, KG_OZ_TRSM, KG_OZ_SYRK, KG_OZ_SYREDUCE,
  KG_OZ_PREPX, KG_OZ_FINALIZE,
  // grouped tensor-core sketch, param = 2 precision + (MT - 1)
  KG_TC_SKETCH
};

constexpr int kSideStreams = 8;

// Emulated-FP64 scratch of one problem (in the batch workspace).
struct OzWs {
  SyrkOzPlan sp;
  SketchOzPlan kp;
  uint32_t* colhi;
  long long* part;
  uint32_t* tcole;
  unsigned char* trd;
  uint32_t* oze;
  unsigned char* ozx;
  uint64_t seed;
};

struct Launch {
  int kind, level, param, off, cnt;
};

struct Tuning {
  int64_t rows_per_split = 4096;
  int64_t rows_per_chunk = 8192;
  int64_t oz_rows_per_slab = 0;   // emulated Gram and check: rows per partial (0: chosen per problem)
};

}  // namespace

struct mrcqr_batched_plan_s {
  int count = 0;
  int max_s = 1;
  bool async_ws = false;
  bool use_graph = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  Prob* d_probs = nullptr;
  int4* d_items = nullptr;
  std::vector<Prob> probs;   // host copy (device pointers inside)
  std::vector<int4> items;
  std::vector<Launch> launches;
  std::vector<unsigned char> maps;    // TMA maps of every A (slabs of 64 and 32 rows), host copy
  size_t maps_off = 0;
  Tuning tuning;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
  bool emu = true;                    // emulated-FP64 heavy phases
  bool oz_grouped = true;             // ... as grouped persistent launches (else per problem on side streams)
  std::vector<OzWs> oz;               // per problem (emu)
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSideStreams] = {};
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, Tuning> g_tune_cache;
bool g_tune_loaded = false;

std::string signature(int count, const int64_t* m, const int64_t* n) {
  // shape histogram: count of problems per (n, floor(log2 m))
  std::map<std::pair<int64_t, int>, int> h;
  for (int i = 0; i < count; ++i) {
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= m[i]) ++lg;
    h[{n[i], lg}]++;
  }
  std::ostringstream os;
  for (auto& kv : h) os << kv.first.first << "x" << kv.first.second << ":" << kv.second << ";";
  return os.str();
}

void load_tune_file() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = getenv("MRCQR_TUNE_CACHE");
  if (!f) return;
  std::ifstream in(f);
  std::string key;
  int64_t a, b, c;
  while (in >> key >> a >> b >> c) g_tune_cache[key] = Tuning{a, b, c};
}

void save_tune_file() {
  const char* f = getenv("MRCQR_TUNE_CACHE");
  if (!f) return;
  std::ofstream out(f);
  for (auto& kv : g_tune_cache)
    out << kv.first << " " << kv.second.rows_per_split << " " << kv.second.rows_per_chunk << " "
        << kv.second.oz_rows_per_slab << "\n";
}

int ladder(int p, bool escalate, int* lv) {
  int k = 0;
  lv[k++] = p;
  if (escalate) {
    if (p == P_FP16 || p == P_BF16) lv[k++] = P_FP32;
    if (p != P_FP64) lv[k++] = P_FP64;
  }
  for (int i = k; i < kMaxLevels; ++i) lv[i] = P_FP64;
  return k;
}

// Per-problem workspace layout and work lists for the given tuning.
void build(mrcqr_batched_plan_s& pl, int count, const int64_t* m, const int64_t* n, const double* const* A,
           const int64_t* lda, double* const* Q, const int64_t* ldq, double* const* R, const int* prec,
           const uint64_t* seeds, int32_t* status, int check, bool escalate, double tol, int tf, size_t* ws_bytes) {
  pl.count = count;
  pl.probs.assign(count, Prob{});
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  std::vector<std::array<size_t, 14>> offs(count);
  pl.max_s = 1;
  int max_levels = 1;
  for (int i = 0; i < count; ++i) {
    Prob& P = pl.probs[i];
    P.A = A[i];
    P.Q = Q[i];
    P.R = R[i];
    P.lda = lda[i];
    P.ldq = ldq[i];
    P.ldr = n[i];
    P.m = m[i];
    P.n = (int)n[i];
    P.tf = tf;
    P.bins = 2 * P.n;
    P.s = tf == T_RFFT_REIM ? 2 * P.bins : P.bins;
    P.npad = (P.n + 31) / 32 * 32;
    P.rows_per_chunk = pl.tuning.rows_per_chunk;
    P.chunks = (int)((P.m + P.rows_per_chunk - 1) / P.rows_per_chunk);
    P.rows_per_split = pl.tuning.rows_per_split;
    P.splits = (int)((P.m + P.rows_per_split - 1) / P.rows_per_split);
    const int tn = syrk_tile_for(P.n);
    P.ntile_syrk = (P.n + tn - 1) / tn;
    P.check = check;
    P.nlevels = ladder(prec[i], escalate, P.lvl_prec);
    P.key = seed_key(seeds[i]);
    P.tol = tol;
    P.status = status + i;
    pl.max_s = std::max(pl.max_s, P.s);
    max_levels = std::max(max_levels, P.nlevels);
    auto& f = offs[i];
    const size_t nn = (size_t)P.n * P.n;
    f[0] = take(sizeof(Ctl));
    f[1] = take(sizeof(uint32_t) * P.s);
    f[2] = take(sizeof(double) * (size_t)(P.m + 1));
    f[3] = take(0);   // (unused slot)
    f[4] = take(sizeof(double) * (size_t)P.chunks * P.s * P.n);
    f[5] = take(sizeof(double) * (size_t)P.s * P.n);
    f[6] = take(sizeof(double) * (size_t)P.s * P.n);
    f[7] = take(sizeof(double) * nn);
    f[8] = take(sizeof(double) * (size_t)P.n * P.npad);
    f[9] = take(sizeof(double) * P.npad);
    f[10] = take(sizeof(double) * (size_t)P.splits * nn);
    f[11] = take(sizeof(double) * nn);
    f[12] = take(sizeof(double) * (size_t)P.n * P.npad);
    f[13] = take(sizeof(double) * nn);
  }
  std::vector<std::array<size_t, 6>> ozoff(pl.emu ? count : 0);
  pl.oz.assign(pl.emu ? count : 0, OzWs{});
  for (int i = 0; i < (pl.emu ? count : 0); ++i) {
    const Prob& P = pl.probs[i];
    OzWs& z = pl.oz[i];
    z.sp = syrk_oz_plan(P.m, P.n, pl.tuning.oz_rows_per_slab);
    z.kp = sketch_oz_plan(P.m, P.n, P.s);
    z.seed = seeds[i];
    auto& g = ozoff[i];
    g[0] = take(syrk_oz_colhi_bytes(P.n));
    g[1] = take(std::max(syrk_oz_part_bytes(z.sp), sketch_oz_part_bytes(z.kp)));
    g[2] = take(trsm_oz_cole_bytes(P.n));
    g[3] = take(trsm_oz_rd_bytes(P.n));
    g[4] = take(sizeof(uint32_t) * (size_t)oz_x_cols(P.n));
    g[5] = take(oz_xs_bytes(P.n));
  }
  const size_t probs_off = take(sizeof(Prob) * (size_t)count);
  const size_t map_bytes = sketch_tc_map_bytes();
  pl.maps_off = take(2 * map_bytes * (size_t)count);
  pl.maps.assign(2 * map_bytes * (size_t)count, 0);
  std::vector<char> maps_ok(count, 0), tc_ok(count, 0);   // TMA maps of A; tensor-core sketch (maps or plain loads)
  for (int i = 0; i < count; ++i) {
    const Prob& P = pl.probs[i];
    maps_ok[i] = sketch_tc_encode(64, P.A, P.lda, P.m, P.n, pl.maps.data() + (2 * i) * map_bytes) &&
                 sketch_tc_encode(32, P.A, P.lda, P.m, P.n, pl.maps.data() + (2 * i + 1) * map_bytes);
    tc_ok[i] = sketch_tc_eligible(P_FP16, P.A, P.lda);
  }
  // work lists
  pl.items.clear();
  pl.launches.clear();
  auto add = [&](int kind, int level, int param, const std::vector<int4>& v) {
    if (v.empty()) return;
    pl.launches.push_back(Launch{kind, level, param, (int)pl.items.size(), (int)v.size()});
    pl.items.insert(pl.items.end(), v.begin(), v.end());
  };
  auto blocks = [](int64_t x, int64_t b) { return (int)((x + b - 1) / b); };
  auto per_problem = [&](int kind, int level, const std::vector<int>& which) {   // fork, one entry each, join
    if (which.empty()) return;
    pl.launches.push_back(Launch{K_FORK, level, 0, 0, 0});
    for (int i : which) pl.launches.push_back(Launch{kind, level, i, 0, 0});
    pl.launches.push_back(Launch{K_JOIN, level, 0, 0, 0});
  };
  pl.launches.push_back(Launch{K_INIT, 0, 0, 0, count});
  {
    std::vector<int4> v, c;
    for (int i = 0; i < count; ++i) {
      v.push_back(make_int4(i, 0, 0, 0));
      for (int b = 0; b < blocks(pl.probs[i].m + 1, 256); ++b) c.push_back(make_int4(i, b, 0, 0));
    }
    add(K_SAMPLE, 0, 0, v);
    add(K_COSTAB, 0, 0, c);
  }
  for (int L = 0; L < max_levels; ++L) {
    std::vector<int> live;
    for (int i = 0; i < count; ++i)
      if (pl.probs[i].nlevels > L) live.push_back(i);
    std::vector<int> oz_sk;   // problems whose sketch at this level is the emulated FP64 one
    for (int pr = P_FP16; pr <= P_FP64; ++pr) {
      std::vector<int4> v, tcv[2];
      for (int i : live) {
        const Prob& P = pl.probs[i];
        if (P.lvl_prec[L] != pr) continue;
        if (pl.emu && pr == P_FP64) {
          oz_sk.push_back(i);
          continue;
        }
        if (tc_ok[i] && pr != P_FP64) {   // tensor cores: 128 or 256 sampled rows per tile
          const int mt = P.s > 128 ? 2 : 1;
          std::vector<int4>& t = tcv[mt - 1];
          for (int c = 0; c < P.chunks; ++c)
            for (int a = 0; a < blocks(P.s, 128 * mt); ++a)
              for (int b = 0; b < blocks(P.n, 64); ++b) t.push_back(make_int4(i, c, a, b));
          continue;
        }
        for (int c = 0; c < P.chunks; ++c)
          for (int a = 0; a < blocks(P.s, 64); ++a)
            for (int b = 0; b < blocks(P.n, 64); ++b) v.push_back(make_int4(i, c, a, b));
      }
      add(K_SKETCH, L, pr, v);
      add(KG_TC_SKETCH, L, 2 * pr, tcv[0]);
      add(KG_TC_SKETCH, L, 2 * pr + 1, tcv[1]);
    }
    if (pl.oz_grouped) {
      std::vector<int4> ch, sk, rd;
      for (int i : oz_sk) {
        const Prob& P = pl.probs[i];
        const OzWs& z = pl.oz[i];
        for (int j = 0; j < (P.n + 127) / 128 * 128; ++j) ch.push_back(make_int4(i, j, 0, 0));
        for (int t = 0; t < z.kp.mblocks * z.kp.ntiles * z.kp.slabs; ++t) sk.push_back(make_int4(i, t, 0, 0));
        for (int b = 0; b < blocks((int64_t)P.s * P.n, 256); ++b) rd.push_back(make_int4(i, b, 0, 0));
      }
      add(KG_OZ_COLHI, L, 0, ch);
      add(KG_OZ_SKETCH, L, 0, sk);
      add(KG_OZ_SKREDUCE, L, 0, rd);
    } else {
      per_problem(K_OZ_SKETCH, L, oz_sk);
    }
    std::vector<int4> red, q32, q64, tr, gr, one, ti, rm, fi;
    for (int i : live) {
      const Prob& P = pl.probs[i];
      if (!(pl.emu && P.lvl_prec[L] == P_FP64))
        for (int b = 0; b < blocks((int64_t)P.s * P.n, 256); ++b) red.push_back(make_int4(i, b, 0, 0));
      (P.lvl_prec[L] == P_FP64 ? q64 : q32).push_back(make_int4(i, 0, 0, 0));
      for (int b = 0; b < blocks(P.m, 128); ++b) tr.push_back(make_int4(i, b, 0, 0));
      for (int b = 0; b < blocks((int64_t)P.n * P.n, 256); ++b) gr.push_back(make_int4(i, b, 0, 0));
      one.push_back(make_int4(i, 0, 0, 0));
      for (int b = 0; b < blocks(P.npad, 64); ++b) ti.push_back(make_int4(i, b, 0, 0));
      for (int b = 0; b < blocks(P.m, 128); ++b) fi.push_back(make_int4(i, b, 0, 0));
    }
    rm = gr;
    add(K_SKREDUCE, L, 0, red);
    add(K_SQR, L, 0, q32);
    add(K_SQR, L, 1, q64);
    // emulated-FP64 stage 2 work lists (grouped form)
    std::vector<int4> z_rs, z_pr, z_tr, z_sy, z_gr, z_px, z_fi;
    if (pl.emu && pl.oz_grouped)
      for (int i : live) {
        const Prob& P = pl.probs[i];
        const OzWs& z = pl.oz[i];
        for (int b = 0; b < blocks(P.n, 8); ++b) z_rs.push_back(make_int4(i, b, 0, 0));
        for (int c = 0; c < (P.n + 15) / 16 * 16; ++c) z_pr.push_back(make_int4(i, c, 0, 0));
        for (int b = 0; b < blocks(P.m, 128); ++b) z_tr.push_back(make_int4(i, b, 0, 0));
        for (int t = 0; t < z.sp.ntiles * z.sp.slabs; ++t) z_sy.push_back(make_int4(i, t, 0, 0));
        for (int b = 0; b < blocks((int64_t)P.n * P.n, 256); ++b) z_gr.push_back(make_int4(i, b, 0, 0));
        for (int j = 0; j < oz_x_cols(P.n); ++j) z_px.push_back(make_int4(i, j, 0, 0));
        for (int b = 0; b < blocks(P.m, 128); ++b) z_fi.push_back(make_int4(i, b, 0, 0));
      }
    if (pl.emu && pl.oz_grouped) {   // W = A R_s^{-1} (folding W's column maxima), G = W^T W
      add(KG_OZ_ROWSCALE, L, 0, z_rs);
      add(KG_OZ_PREPR, L, 0, z_pr);
      add(KG_OZ_TRSM, L, 0, z_tr);
      add(KG_OZ_SYRK, L, 0, z_sy);
      add(KG_OZ_SYREDUCE, L, 0, z_gr);
    } else if (pl.emu) {
      per_problem(K_OZ_STAGE2A, L, live);   // W = A R_s^{-1}, G = W^T W
    } else {
      add(K_TRSM, L, 0, tr);
      for (int tn : {16, 32, 64}) {
        std::vector<int4> v;
        for (int i : live) {
          const Prob& P = pl.probs[i];
          if (syrk_tile_for(P.n) != tn) continue;
          const int tiles = P.ntile_syrk * (P.ntile_syrk + 1) / 2;
          for (int sp = 0; sp < P.splits; ++sp)
            for (int t = 0; t < tiles; ++t) v.push_back(make_int4(i, t, sp, 0));
        }
        add(K_SYRK, L, tn, v);
      }
      add(K_GREDUCE, L, 0, gr);
    }
    add(K_CHOL, L, 0, one);
    add(K_TRINV, L, 0, ti);
    add(K_RMUL, L, 0, rm);
    if (pl.emu && pl.oz_grouped) {   // Q = W R_c^{-1} (folding Q's column maxima), E = Q^T Q
      add(KG_OZ_PREPX, L, 0, z_px);
      add(KG_OZ_FINALIZE, L, 0, z_fi);
      if (check) {
        add(KG_OZ_SYRK, L, 1, z_sy);
        add(KG_OZ_SYREDUCE, L, 1, z_gr);
      }
    } else if (pl.emu) {
      per_problem(K_OZ_STAGE2B, L, live);   // Q = W R_c^{-1}, E = Q^T Q
    } else {
      add(K_FINALIZE, L, 0, fi);
    }
    if (check && !pl.emu) {
      for (int tn : {16, 32, 64}) {
        std::vector<int4> v;
        for (int i : live) {
          const Prob& P = pl.probs[i];
          if (syrk_tile_for(P.n) != tn) continue;
          const int tiles = P.ntile_syrk * (P.ntile_syrk + 1) / 2;
          for (int sp = 0; sp < P.splits; ++sp)
            for (int t = 0; t < tiles; ++t) v.push_back(make_int4(i, t, sp, 0));
        }
        add(K_CHECK, L, tn, v);
      }
      add(K_EREDUCE, L, 0, gr);
    }
    add(K_JUDGE, L, 0, one);
  }
  pl.launches.push_back(Launch{K_PUBLISH, 0, 0, 0, count});
  const size_t items_off = take(sizeof(int4) * std::max<size_t>(1, pl.items.size()));
  *ws_bytes = o;
  // resolve device pointers relative to the workspace base stored in pl.ws
  char* base = static_cast<char*>(pl.ws);
  for (int i = 0; i < count; ++i) {
    Prob& P = pl.probs[i];
    auto& f = offs[i];
    P.ctl = reinterpret_cast<Ctl*>(base + f[0]);
    P.idx = reinterpret_cast<uint32_t*>(base + f[1]);
    P.tab = reinterpret_cast<double*>(base + f[2]);
    P.ypart = reinterpret_cast<double*>(base + f[4]);
    P.y = reinterpret_cast<double*>(base + f[5]);
    P.sqrw = base + f[6];
    P.rs = reinterpret_cast<double*>(base + f[7]);
    P.rst = reinterpret_cast<double*>(base + f[8]);
    P.rinv = reinterpret_cast<double*>(base + f[9]);
    P.gpart = reinterpret_cast<double*>(base + f[10]);
    P.rc = reinterpret_cast<double*>(base + f[11]);
    P.xt = reinterpret_cast<double*>(base + f[12]);
    P.e = reinterpret_cast<double*>(base + f[13]);
  }
  for (int i = 0; i < (int)pl.oz.size(); ++i) {
    OzWs& z = pl.oz[i];
    auto& g = ozoff[i];
    z.colhi = reinterpret_cast<uint32_t*>(base + g[0]);
    z.part = reinterpret_cast<long long*>(base + g[1]);
    z.tcole = reinterpret_cast<uint32_t*>(base + g[2]);
    z.trd = reinterpret_cast<unsigned char*>(base + g[3]);
    z.oze = reinterpret_cast<uint32_t*>(base + g[4]);
    z.ozx = reinterpret_cast<unsigned char*>(base + g[5]);
  }
  for (int i = 0; i < (int)pl.oz.size(); ++i) {
    Prob& P = pl.probs[i];
    const OzWs& z = pl.oz[i];
    P.oz_sp = z.sp;
    P.oz_kp = z.kp;
    P.oz_colhi = z.colhi;
    P.oz_part = z.part;
    P.oz_cole = reinterpret_cast<int*>(z.tcole);
    P.oz_rd = z.trd;
    P.oz_xe = z.oze;
    P.oz_xs = z.ozx;
  }
  for (int i = 0; i < count; ++i) {
    pl.probs[i].tmap64 = maps_ok[i] ? base + pl.maps_off + (2 * i) * map_bytes : nullptr;
    pl.probs[i].tmap32 = maps_ok[i] ? base + pl.maps_off + (2 * i + 1) * map_bytes : nullptr;
  }
  pl.d_probs = reinterpret_cast<Prob*>(base + probs_off);
  pl.d_items = reinterpret_cast<int4*>(base + items_off);
}

// The emulated-FP64 kernels of one problem's heavy phase (its control block
// makes them return at once unless the problem is active at this level).
void enqueue_oz(const mrcqr_batched_plan_s& pl, int kind, int level, int i, cudaStream_t st) {
  const Prob& P = pl.probs[i];
  const OzWs& z = pl.oz[i];
  switch (kind) {
    case K_OZ_SKETCH:
      launch_sketch_oz(P.m, P.n, P.s, P.A, P.lda, P.idx, P.tab, z.seed, z.kp, z.colhi, z.part, P.y, P.ctl, level, st,
                       P.tf);
      break;
    case K_OZ_STAGE2A:
      launch_trsm_oz(P.m, P.n, P.A, P.lda, P.rst, P.rinv, z.tcole, z.trd, P.Q, P.ldq, P.ctl, level, st, z.colhi);
      launch_syrk_oz(P.m, P.n, P.Q, P.ldq, z.sp, z.colhi, z.part, P.rc, P.ctl, level, st, true);
      break;
    case K_OZ_STAGE2B:
      launch_finalize_oz(P.m, P.n, P.Q, P.ldq, P.xt, z.oze, z.ozx, P.ctl, level, st, P.check ? z.colhi : nullptr);
      if (P.check) launch_syrk_oz(P.m, P.n, P.Q, P.ldq, z.sp, z.colhi, z.part, P.e, P.ctl, level, st, true);
      break;
  }
}

void enqueue(mrcqr_batched_plan_s& pl, cudaStream_t st) {
  const uint64_t c0 = mrcqr_launch_count();
  int rr = 0;   // next side stream
  for (const Launch& L : pl.launches) {
    Group g{pl.d_probs, pl.d_items + L.off, L.cnt};
    switch (L.kind) {
      case K_FORK:
        cudaEventRecord(pl.fork_ev, st);
        for (int k = 0; k < kSideStreams; ++k) cudaStreamWaitEvent(pl.side[k], pl.fork_ev, 0);
        rr = 0;
        break;
      case K_JOIN:
        for (int k = 0; k < kSideStreams; ++k) {
          cudaEventRecord(pl.join_ev[k], pl.side[k]);
          cudaStreamWaitEvent(st, pl.join_ev[k], 0);
        }
        break;
      case K_OZ_SKETCH:
      case K_OZ_STAGE2A:
      case K_OZ_STAGE2B:
        enqueue_oz(pl, L.kind, L.level, L.param, pl.side[rr]);
        rr = (rr + 1) % kSideStreams;
        break;
      case K_INIT: launch_g_init(Group{pl.d_probs, nullptr, L.cnt}, st); break;
      case K_SAMPLE: launch_g_sample(g, pl.max_s, st); break;
      case K_COSTAB: launch_g_costab(g, st); break;
      case K_SKETCH: launch_g_sketch(g, L.param, L.level, st); break;
      case K_SKREDUCE: launch_g_sketch_reduce(g, L.level, st); break;
      case K_SQR: launch_g_sketch_qr(g, L.param == 1, L.level, st); break;
      case K_TRSM: launch_g_trsm(g, L.level, st); break;
      case K_SYRK: launch_g_syrk(g, L.param, false, L.level, st); break;
      case K_GREDUCE: launch_g_reduce(g, false, L.level, st); break;
      case K_CHOL: launch_g_chol(g, L.level, st); break;
      case K_TRINV: launch_g_trinv(g, L.level, st); break;
      case K_RMUL: launch_g_rmul(g, L.level, st); break;
      case K_FINALIZE: launch_g_finalize(g, L.level, st); break;
      case K_CHECK: launch_g_syrk(g, L.param, true, L.level, st); break;
      case K_EREDUCE: launch_g_reduce(g, true, L.level, st); break;
      case K_JUDGE: launch_g_judge(g, L.level, st); break;
      case K_PUBLISH: launch_g_publish(Group{pl.d_probs, nullptr, L.cnt}, st); break;
      case KG_OZ_COLHI: launch_g_oz_colhi(g, L.level, st); break;
      case KG_OZ_SKETCH: launch_g_oz_sketch(g, L.level, st); break;
      case KG_OZ_SKREDUCE: launch_g_oz_sketch_reduce(g, L.level, st); break;
      case KG_OZ_ROWSCALE: launch_g_oz_row_scale(g, L.level, st); break;
      case KG_OZ_PREPR: launch_g_oz_prep_r(g, L.level, st); break;
      case KG_OZ_TRSM: launch_g_oz_trsm(g, L.level, st); break;
      case KG_TC_SKETCH: launch_g_sketch_tc(g, L.param / 2, L.param % 2 + 1, L.level, st); break;
      case KG_OZ_SYRK: launch_g_oz_syrk(g, L.param == 1, L.level, st); break;
      case KG_OZ_SYREDUCE: launch_g_oz_syrk_reduce(g, L.param == 1, L.level, st); break;
      case KG_OZ_PREPX: launch_g_oz_prep_x(g, L.level, st); break;
      case KG_OZ_FINALIZE: launch_g_oz_finalize(g, L.level, st); break;
    }
  }
  pl.kernels = (int)(mrcqr_launch_count() - c0);
}

// Kernels one execute launches (each emulated heavy phase of a problem is
// several kernels: sketch 3; TRSM 3 + Gram 3; finalize 2 + check 3).
int count_kernels(const mrcqr_batched_plan_s& pl) {
  int k = 0;
  for (const Launch& L : pl.launches) {
    switch (L.kind) {
      case K_FORK: case K_JOIN: break;
      case K_OZ_SKETCH: k += 3; break;
      case K_OZ_STAGE2A: k += 6; break;
      case K_OZ_STAGE2B: k += pl.probs[L.param].check ? 5 : 2; break;
      default: k += 1;
    }
  }
  return k;
}

bool make_streams(mrcqr_batched_plan_s& pl) {
  if (cudaEventCreateWithFlags(&pl.fork_ev, cudaEventDisableTiming) != cudaSuccess) return false;
  for (int k = 0; k < kSideStreams; ++k)
    if (cudaStreamCreateWithFlags(&pl.side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl.join_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return false;
  return true;
}

void free_streams(mrcqr_batched_plan_s& pl) {
  for (int k = 0; k < kSideStreams; ++k) {
    if (pl.side[k]) cudaStreamDestroy(pl.side[k]);
    if (pl.join_ev[k]) cudaEventDestroy(pl.join_ev[k]);
    pl.side[k] = nullptr;
    pl.join_ev[k] = nullptr;
  }
  if (pl.fork_ev) cudaEventDestroy(pl.fork_ev);
  pl.fork_ev = nullptr;
}

int validate_batch(int count, const int64_t* m, const int64_t* n, const double* const* A, const int64_t* lda,
                   double* const* Q, const int64_t* ldq, double* const* R, const int* prec, const uint64_t* seeds,
                   int32_t* status) {
  if (count < 1 || !m || !n || !A || !lda || !Q || !ldq || !R || !prec || !seeds || !status) return MRCQR_ERR_INVALID;
  for (int i = 0; i < count; ++i) {
    if (!A[i] || !Q[i] || !R[i]) return MRCQR_ERR_INVALID;
    if (n[i] < 1 || n[i] > 512 || m[i] < 2 * n[i] || m[i] >= (int64_t(1) << 31)) return MRCQR_ERR_INVALID;
    if (lda[i] < m[i] || ldq[i] < m[i]) return MRCQR_ERR_INVALID;
    if (prec[i] < P_FP16 || prec[i] > P_FP64) return MRCQR_ERR_INVALID;
  }
  return MRCQR_OK;
}

// Times one grouped phase of the plan (level 0) with the given tuning.
float time_phase(mrcqr_batched_plan_s& pl, int kind, cudaStream_t st) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // controls must say "active at level 0"
  launch_g_init(Group{pl.d_probs, nullptr, pl.count}, st);
  cudaEventRecord(a, st);
  for (const Launch& L : pl.launches) {
    if (L.kind != kind || L.level != 0) continue;
    Group g{pl.d_probs, pl.d_items + L.off, L.cnt};
    if (kind == K_SYRK) launch_g_syrk(g, L.param, false, 0, st);
    if (kind == K_SKETCH) launch_g_sketch(g, L.param, 0, st);
    if (kind == KG_TC_SKETCH) launch_g_sketch_tc(g, L.param / 2, L.param % 2 + 1, 0, st);
    if (kind == KG_OZ_SYRK && L.param == 0) launch_g_oz_syrk(g, false, 0, st);
  }
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

}  // namespace

namespace {

// async = true: workspace from the stream-ordered allocator on `st` and the
// work lists copied on `st` (one-shot batches); no tuning in that mode.
int plan_create(int count, const int64_t* m, const int64_t* n, const double* const* A, const int64_t* lda,
                double* const* Q, const int64_t* ldq, double* const* R, const int* sketch_prec, const uint64_t* seeds,
                int32_t* status, const mrcqr_batched_opts_t* opts, mrcqr_batched_plan_t* out, bool async,
                cudaStream_t st) {
  if (!out) return MRCQR_ERR_INVALID;
  *out = nullptr;
  int rc = validate_batch(count, m, n, A, lda, Q, ldq, R, sketch_prec, seeds, status);
  if (rc != MRCQR_OK) return rc;
  // sketch transform: 2n sampled rows (DCT) or bins (real FFT: at most floor(m/2) + 1; Re + Im rows <= 8192)
  const int tf = opts ? opts->transform : T_DCT;
  if (tf < T_DCT || tf > T_RFFT_REIM) return MRCQR_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (tf != T_DCT && (2 * n[i] > m[i] / 2 + 1 || (tf == T_RFFT_REIM && 4 * n[i] > 8192))) return MRCQR_ERR_INVALID;
  auto* pl = new mrcqr_batched_plan_s();
  const int check = opts ? (opts->check != 0) : 1;
  const bool escalate = opts ? (opts->escalate != 0) : true;
  const double tol = (opts && opts->ortho_tol > 0) ? opts->ortho_tol : 1e-13;
  pl->use_graph = opts ? (opts->use_graph != 0) : false;
  pl->emu = opts ? (opts->fp64_products == 0) : true;
  pl->oz_grouped = !(opts && opts->oz_per_problem);
  if (!make_streams(*pl)) {
    free_streams(*pl);
    delete pl;
    return MRCQR_ERR_CUDA;
  }
  const std::string sig = signature(count, m, n);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_file();
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) pl->tuning = it->second;
  }
  if (opts && opts->rows_per_split > 0) pl->tuning.rows_per_split = (opts->rows_per_split + 31) / 32 * 32;
  if (opts && opts->rows_per_chunk > 0) pl->tuning.rows_per_chunk = (opts->rows_per_chunk + 63) / 64 * 64;
  size_t bytes = 0;
  const bool tune = opts && opts->autotune && !async;
  pl->async_ws = async;
  Tuning best = pl->tuning;
  build(*pl, count, m, n, A, lda, Q, ldq, R, sketch_prec, seeds, status, check, escalate, tol, tf, &bytes);
  if (tune) {
    // size the workspace for the candidates with the most partials
    for (const Tuning& t : {Tuning{1024, 2048, 4096}, Tuning{1024, 2048, 0}}) {
      size_t b = 0;
      pl->tuning = t;
      build(*pl, count, m, n, A, lda, Q, ldq, R, sketch_prec, seeds, status, check, escalate, tol, tf, &b);
      bytes = std::max(bytes, b);
    }
  }
  if ((async ? cudaMallocAsync(&pl->ws, bytes, st) : cudaMalloc(&pl->ws, bytes)) != cudaSuccess) {
    cudaGetLastError();
    free_streams(*pl);
    delete pl;
    return MRCQR_ERR_ALLOC;
  }
  pl->ws_bytes = bytes;
  auto upload = [&]() -> int {
    size_t dummy = 0;
    build(*pl, count, m, n, A, lda, Q, ldq, R, sketch_prec, seeds, status, check, escalate, tol, tf, &dummy);
    if (dummy > pl->ws_bytes) return MRCQR_ERR_ALLOC;
    if (async) {   // pageable sources: the copies are staged before these calls return
      if (cudaMemcpyAsync(pl->d_probs, pl->probs.data(), sizeof(Prob) * pl->probs.size(), cudaMemcpyHostToDevice,
                          st) != cudaSuccess ||
          cudaMemcpyAsync(static_cast<char*>(pl->ws) + pl->maps_off, pl->maps.data(), pl->maps.size(),
                          cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(pl->d_items, pl->items.data(), sizeof(int4) * pl->items.size(), cudaMemcpyHostToDevice,
                          st) != cudaSuccess)
        return MRCQR_ERR_CUDA;
      return MRCQR_OK;
    }
    if (cudaMemcpy(pl->d_probs, pl->probs.data(), sizeof(Prob) * pl->probs.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(static_cast<char*>(pl->ws) + pl->maps_off, pl->maps.data(), pl->maps.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl->d_items, pl->items.data(), sizeof(int4) * pl->items.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return MRCQR_ERR_CUDA;
    return MRCQR_OK;
  };
  prepare_g_kernels(2 * 512);
  prepare_g_oz_kernels();
  prepare_g_sketch_tc();
  if (tune) {
    cudaStream_t ts;
    cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
    float bt = 1e30f;
    for (int64_t rps : {1024, 2048, 4096, 8192}) {
      pl->tuning = Tuning{rps, 2048, 0};
      if ((rc = upload()) != MRCQR_OK) break;
      time_phase(*pl, K_SYRK, ts);   // warm
      const float t = time_phase(*pl, K_SYRK, ts);
      if (t < bt) { bt = t; best.rows_per_split = rps; }
    }
    bt = 1e30f;
    for (int64_t rpc : {2048, 4096, 8192, 16384}) {
      pl->tuning = Tuning{best.rows_per_split, rpc, 0};
      if ((rc = upload()) != MRCQR_OK) break;
      time_phase(*pl, K_SKETCH, ts);
      time_phase(*pl, KG_TC_SKETCH, ts);
      const float t = time_phase(*pl, K_SKETCH, ts) + time_phase(*pl, KG_TC_SKETCH, ts);
      if (t < bt) { bt = t; best.rows_per_chunk = rpc; }
    }
    if (pl->emu && pl->oz_grouped) {   // the emulated Gram's slab height, on the grouped launch itself
      bt = 1e30f;
      for (int64_t rps : {0, 4096, 16384, 65536}) {
        pl->tuning = Tuning{best.rows_per_split, best.rows_per_chunk, rps};
        if (upload() != MRCQR_OK) continue;
        time_phase(*pl, KG_OZ_SYRK, ts);
        const float t = time_phase(*pl, KG_OZ_SYRK, ts);
        if (t < bt) { bt = t; best.oz_rows_per_slab = rps; }
      }
    }
    cudaStreamDestroy(ts);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[sig] = best;
    save_tune_file();
  }
  pl->tuning = best;
  if (rc == MRCQR_OK) rc = upload();
  if (rc == MRCQR_OK) pl->kernels = count_kernels(*pl);
  if (rc != MRCQR_OK) {
    if (async) cudaFreeAsync(pl->ws, st);
    else cudaFree(pl->ws);
    free_streams(*pl);
    delete pl;
    return rc;
  }
  *out = pl;
  return MRCQR_OK;
}

}  // namespace

extern "C" {

int mrcqr_batched_plan_create(int count, const int64_t* m, const int64_t* n, const double* const* A, const int64_t* lda,
                              double* const* Q, const int64_t* ldq, double* const* R, const int* sketch_prec,
                              const uint64_t* seeds, int32_t* status, const mrcqr_batched_opts_t* opts,
                              mrcqr_batched_plan_t* out) {
  return plan_create(count, m, n, A, lda, Q, ldq, R, sketch_prec, seeds, status, opts, out, false, nullptr);
}

int mrcqr_factor_batched(int count, const int64_t* m, const int64_t* n, const double* const* A, const int64_t* lda,
                         double* const* Q, const int64_t* ldq, double* const* R, const int* sketch_prec,
                         const uint64_t* seeds, int32_t* status, mrcqr_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  mrcqr_batched_plan_t pl = nullptr;
  int rc = plan_create(count, m, n, A, lda, Q, ldq, R, sketch_prec, seeds, status, nullptr, &pl, true, st);
  if (rc != MRCQR_OK) return rc;
  enqueue(*pl, st);
  cudaFreeAsync(pl->ws, st);
  pl->ws = nullptr;
  free_streams(*pl);   // released once their queued work completes
  delete pl;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "mrcqr batched: CUDA error %s\n", cudaGetErrorString(e));
    return MRCQR_ERR_CUDA;
  }
  return MRCQR_OK;
}

int mrcqr_batched_plan_execute(mrcqr_batched_plan_t pl, mrcqr_stream_t stream) {
  if (!pl) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!pl->use_graph) {
    enqueue(*pl, st);
  } else {
    if (!pl->exec) {
      if (cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) != cudaSuccess) return MRCQR_ERR_CUDA;
      if (cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MRCQR_ERR_CUDA;
      enqueue(*pl, pl->cap);
      if (cudaStreamEndCapture(pl->cap, &pl->graph) != cudaSuccess) return MRCQR_ERR_CUDA;
      if (cudaGraphInstantiate(&pl->exec, pl->graph, 0) != cudaSuccess) return MRCQR_ERR_CUDA;
    }
    if (cudaGraphLaunch(pl->exec, st) != cudaSuccess) return MRCQR_ERR_CUDA;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "mrcqr batched: CUDA error %s\n", cudaGetErrorString(e));
    return MRCQR_ERR_CUDA;
  }
  return MRCQR_OK;
}

int mrcqr_batched_plan_info(mrcqr_batched_plan_t pl, int64_t* rows_per_split, int64_t* rows_per_chunk,
                            int32_t* kernels_per_execute, int64_t* workspace_bytes) {
  if (!pl) return MRCQR_ERR_INVALID;
  if (rows_per_split) *rows_per_split = pl->tuning.rows_per_split;
  if (rows_per_chunk) *rows_per_chunk = pl->tuning.rows_per_chunk;
  if (kernels_per_execute) *kernels_per_execute = pl->kernels > 0 ? pl->kernels : (int32_t)pl->launches.size();
  if (workspace_bytes) *workspace_bytes = (int64_t)pl->ws_bytes;
  return MRCQR_OK;
}

int mrcqr_batched_plan_destroy(mrcqr_batched_plan_t pl) {
  if (!pl) return MRCQR_ERR_INVALID;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  free_streams(*pl);
  if (pl->ws) {
    if (pl->async_ws) cudaFreeAsync(pl->ws, nullptr);
    else cudaFree(pl->ws);
  }
  delete pl;
  return MRCQR_OK;
}

}  // extern "C"
