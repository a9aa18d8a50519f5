// Host planner: splits the n qubit levels into passes and lays out each pass's
// tile and stages (see tpd_plan.h).
#include "tpd_planner.h"
#include "tpd_shape.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <memory>
#include <vector>

namespace tpd {

namespace {

struct Level { int c, r; };  // tile bit positions of a level's column and row bit

struct StageChoice {
  std::vector<int> pairs, shfls;  // level indices
};

struct SearchCtx {
  int D, lf, K;
  std::vector<Level> lev;
  double cx, cs;
  // memo over (stage index, remaining-level mask): best cost and choice
  double memo_cost[kMaxStages + 1][1 << kMaxLevels];
  int memo_nst[kMaxStages + 1][1 << kMaxLevels];
  bool memo_done[kMaxStages + 1][1 << kMaxLevels];
  StageChoice memo_choice[kMaxStages + 1][1 << kMaxLevels];
};

bool in(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

// Lanes of stage `si` for a choice: stage 0 uses tile bits 0..4; later stages
// the forced low bits, the shuffles' column bits, then the lowest free bits.
bool stage_lanes(const SearchCtx& c, int si, const StageChoice& ch, std::vector<int>& lanes,
                 std::vector<int>& regs) {
  regs.clear();
  for (int j : ch.pairs) { regs.push_back(c.lev[j].c); regs.push_back(c.lev[j].r); }
  for (int j : ch.shfls) regs.push_back(c.lev[j].r);
  lanes.clear();
  if (si == 0) {
    for (int i = 0; i < kLaneBits; ++i) lanes.push_back(i);
  } else {
    for (int i = 0; i < c.lf; ++i) lanes.push_back(i);
    for (int j : ch.shfls)
      if (!in(lanes, c.lev[j].c)) lanes.push_back(c.lev[j].c);
    for (int b = 0; b < c.D && (int)lanes.size() < kLaneBits; ++b)
      if (!in(lanes, b) && !in(regs, b)) lanes.push_back(b);
  }
  if ((int)lanes.size() != kLaneBits) return false;
  for (int x : regs)
    if (in(lanes, x)) return false;
  for (int j : ch.shfls)
    if (!in(lanes, c.lev[j].c)) return false;
  return (int)regs.size() <= kRegBits;
}

// Cheapest way to finish the levels in `remaining` starting at stage si:
// each stage after the first costs an exchange, each shuffle level its cost.
double search(SearchCtx& c, int si, unsigned remaining, int* nst) {
  if (remaining == 0) { *nst = 0; return 0.0; }
  if (si >= kMaxStages) { *nst = 99; return 1e30; }
  if (c.memo_done[si][remaining]) { *nst = c.memo_nst[si][remaining]; return c.memo_cost[si][remaining]; }
  std::vector<int> rem;
  for (int j = 0; j < c.K; ++j)
    if (remaining & (1u << j)) rem.push_back(j);
  const int R = (int)rem.size();
  int total = 1;
  for (int i = 0; i < R; ++i) total *= 3;
  double best = 1e30;
  int best_nst = 99;
  StageChoice best_ch;
  std::vector<int> lanes, regs;
  for (int code = 1; code < total; ++code) {  // per level: 0 later, 1 pair, 2 shuffle
    StageChoice ch;
    int x = code;
    for (int i = 0; i < R; ++i, x /= 3) {
      if (x % 3 == 1) ch.pairs.push_back(rem[i]);
      else if (x % 3 == 2) ch.shfls.push_back(rem[i]);
    }
    if ((int)ch.pairs.size() > 2) continue;
    if (2 * (int)ch.pairs.size() + (int)ch.shfls.size() > kRegBits) continue;
    if (!stage_lanes(c, si, ch, lanes, regs)) continue;
    unsigned done = 0;
    for (int j : ch.pairs) done |= 1u << j;
    for (int j : ch.shfls) done |= 1u << j;
    int sub_nst = 0;
    const double sub = search(c, si + 1, remaining & ~done, &sub_nst);
    const double cost = (si > 0 ? c.cx : 0.0) + c.cs * (double)ch.shfls.size() + sub;
    if (cost < best - 1e-9 || (cost < best + 1e-9 && sub_nst + 1 < best_nst)) {
      best = cost; best_nst = sub_nst + 1; best_ch = ch;
    }
  }
  c.memo_done[si][remaining] = true;
  c.memo_cost[si][remaining] = best;
  c.memo_nst[si][remaining] = best_nst;
  c.memo_choice[si][remaining] = best_ch;
  *nst = best_nst;
  return best;
}

// Tile mask of a pass: the 2K level bits plus the D-2K lowest column bits
// outside the group, then the lowest row bits.
std::vector<int> tile_bits(int n, int b, int K, int D) {
  std::vector<int> t;
  for (int j = 0; j < K; ++j) { t.push_back(b + j); t.push_back(n + b + j); }
  for (int g = 0; g < 2 * n && (int)t.size() < D; ++g)
    if (!in(t, g)) t.push_back(g);
  std::sort(t.begin(), t.end());
  return t;
}

bool build_pass(int n, int b, int K, int D, int lf, double cs, PassDesc* pd, std::string* err,
                double* cost_out = nullptr) {
  std::memset(pd, 0, sizeof(*pd));
  if (K < 1 || K > kMaxLevels || D < kMinTileBits || D > kMaxTileBits || 2 * K > D || D > 2 * n ||
      b < 0 || b + K > n) {
    if (err) *err = "invalid pass shape";
    return false;
  }
  std::vector<int> t = tile_bits(n, b, K, D);
  pd->n = n; pd->D = D; pd->K = K; pd->b = b;
  for (int i = 0; i < D; ++i) pd->gbit[i] = (int8_t)t[i];
  std::vector<int> rest;
  for (int g = 0; g < 2 * n; ++g)
    if (!in(t, g)) rest.push_back(g);
  pd->nrest = (int)rest.size();
  for (int j = 0; j < pd->nrest; ++j) pd->rest_gbit[j] = (int8_t)rest[j];
  pd->ntiles = 1ll << pd->nrest;

  std::unique_ptr<SearchCtx> cp(new SearchCtx());
  SearchCtx& c = *cp;
  for (int si = 0; si <= kMaxStages; ++si)
    for (int m = 0; m < (1 << kMaxLevels); ++m) c.memo_done[si][m] = false;
  c.D = D; c.lf = lf; c.K = K;
  for (int j = 0; j < K; ++j) {
    Level L;
    L.c = (int)(std::find(t.begin(), t.end(), b + j) - t.begin());
    L.r = (int)(std::find(t.begin(), t.end(), n + b + j) - t.begin());
    c.lev.push_back(L);
  }
  // class bits (see PassDesc::cls_w): column-type tile bits in ascending
  // order, each level's row bit on its column's class bit
  {
    std::vector<int> pos(D, -1);
    int next = 0;
    for (int i = 0; i < D; ++i) {
      bool row = false;
      for (const Level& L : c.lev) row |= L.r == i;
      if (!row) pos[i] = next++;
    }
    for (const Level& L : c.lev) pos[L.r] = pos[L.c];
    for (int i = 0; i < D; ++i) pd->cls_w[i] = 1 << pos[i];
  }
  c.cx = 2.0; c.cs = cs;
  int nst = 0;
  const double cost = search(c, 0, (1u << K) - 1, &nst);
  if (cost >= 1e29) {
    if (err) *err = "no stage plan";
    return false;
  }
  if (cost_out) *cost_out = cost;
  std::vector<StageChoice> chosen;
  unsigned remaining = (1u << K) - 1;
  for (int si = 0; remaining; ++si) {
    const StageChoice& ch = c.memo_choice[si][remaining];
    chosen.push_back(ch);
    for (int j : ch.pairs) remaining &= ~(1u << j);
    for (int j : ch.shfls) remaining &= ~(1u << j);
  }
  pd->nstage = (int)chosen.size();
  std::vector<int> lanes, regs;
  for (int si = 0; si < pd->nstage; ++si) {
    const StageChoice& ch = chosen[si];
    stage_lanes(c, si, ch, lanes, regs);
    Stage& st = pd->st[si];
    std::vector<bool> used(D, false);
    for (int x : lanes) used[x] = true;
    for (int x : regs) used[x] = true;
    // fillers: the highest unused bits
    for (int bit = D - 1; bit >= 0 && (int)regs.size() < kRegBits; --bit)
      if (!used[bit]) { regs.push_back(bit); used[bit] = true; }
    std::vector<int> warps;
    for (int bit = 0; bit < D; ++bit)
      if (!used[bit]) warps.push_back(bit);
    std::sort(lanes.begin(), lanes.end());
    for (int i = 0; i < kRegSlots; ++i) st.reg[i] = (int8_t)(i < kRegBits ? regs[i] : 0);
    for (int i = 0; i < kLaneBits; ++i) st.lane[i] = (int8_t)lanes[i];
    for (int i = 0; i < (int)warps.size(); ++i) st.warp[i] = (int8_t)warps[i];
    st.npair = (int8_t)ch.pairs.size();
    st.nshfl = (int8_t)ch.shfls.size();
    for (int s = 0; s < st.nshfl; ++s) {
      const int cb = c.lev[ch.shfls[s]].c;
      st.shfl_lane[s] = (int8_t)(std::find(lanes.begin(), lanes.end(), cb) - lanes.begin());
    }
  }
  return true;
}

void set_next(PassDesc* cur, const PassDesc& nxt) {
  std::vector<int> rest_next(nxt.rest_gbit, nxt.rest_gbit + nxt.nrest);
  auto w = [&](int g) -> long long {
    auto it = std::find(rest_next.begin(), rest_next.end(), g);
    if (it == rest_next.end()) return 0;
    return 1ll << (int)(it - rest_next.begin());
  };
  cur->has_next = 1;
  for (int i = 0; i < cur->D; ++i) cur->next_w[i] = (int32_t)w(cur->gbit[i]);
  for (int j = 0; j < cur->nrest; ++j) cur->next_rest_w[j] = w(cur->rest_gbit[j]);
}

// Index, in the previous pass's binary-point array, of an element's class
// there, as XOR weights of the current pass's tile and tile-id bits: a global
// bit that is a tile-id bit j of the previous pass contributes bit
// (D' - K') + j (the tile id above the class bits), one that is a tile bit i
// there its class bit cls_w[i].
void set_src(PassDesc* cur, const PassDesc& prv) {
  const int ncls_bits = prv.D - prv.K;
  auto w = [&](int g) -> uint32_t {
    for (int j = 0; j < prv.nrest; ++j)
      if (prv.rest_gbit[j] == g) return 1u << (ncls_bits + j);
    for (int i = 0; i < prv.D; ++i)
      if (prv.gbit[i] == g) return (uint32_t)prv.cls_w[i];
    return 0u;
  };
  cur->has_prev = 1;
  for (int i = 0; i < cur->D; ++i) cur->src_w[i] = w(cur->gbit[i]);
  for (int j = 0; j < cur->nrest; ++j) cur->src_rest_w[j] = w(cur->rest_gbit[j]);
}

}  // namespace

int arith_elem_bytes(int dtype, int precision) {
  if (dtype == 0) return 16;               // fixed int64 pair or double2
  return precision >= 2 ? 16 : 8;          // compensated hi/lo pairs, fixed-point int64 pairs in registers
}

bool build_plan(int n, int dtype, int precision, int tile_bits_opt, int max_levels_opt, Plan* plan,
                std::string* err) {
  std::memset(plan, 0, sizeof(*plan));
  plan->n = n;
  plan->elem_bytes = arith_elem_bytes(dtype, precision);
  if (n < 1 || n > kMaxQubits) {
    if (err) *err = "n out of range";
    return false;
  }
  if (2 * n < kMinTileBits) {  // whole matrix in one CTA
    plan->npass = 0;
    return true;
  }
  // Low tile bits always on lanes: 3 (complex128: 128-byte runs; complex64:
  // 64-byte runs, which let 5-level passes fit in 2^13-element tiles and save
  // a pass: measured on GB300 at n = 15, fixed point 37.3 -> 31.3 ms, plain
  // 12.24 -> 11.66 ms, equal at n = 13 and 14).  The compensated complex64
  // form keeps 4 (128-byte runs): its passes slow down more with the shorter
  // runs than a pass saves (20.8 against 22.2 ms at n = 15).
  const int lf = (dtype == 1 && precision == 2) ? 4 : 3;
  const double cs = plan->elem_bytes == 16 ? 1.0 : 0.5;    // shuffle cost per level
  // 2^12-element tiles by default: two CTAs of 256 threads fit an SM; 2^13
  // (512 threads, one CTA per SM) only where it saves a pass (below)
  int dmax = tile_bits_opt ? tile_bits_opt : 12;
  dmax = std::min(dmax, 2 * n);
  int kcap = max_levels_opt ? max_levels_opt : kMaxLevels;
  auto kmax_for = [&](int D) { return std::max(1, std::min({(D - lf) / 2, kcap, kMaxLevels})); };
  // A pass over 2^13-element tiles (the 5-level passes) runs ~1.6x longer than
  // one over 2^12 on GB300 (128-byte runs; measured 3.2-4.6 against 5.1-5.7
  // TB/s), so it counts as 1.6 passes when plans are compared.
  constexpr double kWeightD13 = 1.6;
  auto weight = [&](const std::vector<std::pair<int, int>>& g) {
    double w = 0.0;
    for (const auto& kd : g) w += kd.second > 12 ? kWeightD13 : 1.0;
    return w;
  };
  // passes for a first pass of k0 levels: the rest split evenly over as few
  // passes as possible (2^13-element tiles only where that weighs less)
  auto groups_for = [&](int k0) {
    std::vector<std::pair<int, int>> g;  // (K, D)
    g.push_back({k0, dmax});
    const int rem = n - k0;
    if (rem > 0) {
      // where 2^13-element tiles are chosen, only the passes that need them
      // get them; the others take the smallest tile with 128-byte runs, 2K +
      // lf bits (measured on GB300, n = 15 last pass of 4 levels: 9.72 ms
      // with 2^13, 8.09 ms with 2^12, 7.28 ms with 2^11 elements)
      auto split = [&](int D1) {
        std::vector<std::pair<int, int>> r;
        const int m = (rem + kmax_for(D1) - 1) / kmax_for(D1);
        const int base = rem / m, extra = rem % m;
        for (int i = 0; i < m; ++i) {
          const int K = base + (i < extra ? 1 : 0);
          const int Dsmall = std::max(kMinTileBits, 2 * K + lf);
          r.push_back({K, (D1 > dmax && K <= kmax_for(dmax)) ? Dsmall : D1});
        }
        return r;
      };
      std::vector<std::pair<int, int>> rest = split(dmax);
      if (!tile_bits_opt && dmax < kMaxTileBits && 2 * n >= dmax + 1) {
        std::vector<std::pair<int, int>> r13 = split(dmax + 1);
        if (weight(r13) < weight(rest) - 1e-9) rest = r13;
      }
      g.insert(g.end(), rest.begin(), rest.end());
    }
    // complex128: a middle pass (int64 in and out) on the smallest tile with
    // 128-byte runs (2K + lf bits: 2^11 elements for 4 levels, four CTAs of
    // 128 threads per SM instead of two of 256) -- measured on GB300 with the
    // compiled layouts, n = 14 middle pass 1.550 -> 1.397 ms, n = 13 0.374 ->
    // 0.340 ms, n = 16 25.9 / 26.9 -> 21.5 / 24.7 ms; the first and last
    // passes keep 2^12 (the last one ran 3-4 % slower on 2^11), complex64
    // keeps 2^12 (plain n = 14 passes 0.62 / 0.64 -> 0.68 / 0.74 ms)
    if (dtype == 0 && !tile_bits_opt)
      for (size_t i = 1; i + 1 < g.size(); ++i) {
        const int Dsmall = std::max(kMinTileBits, 2 * g[i].first + lf);
        if (Dsmall < g[i].second) g[i].second = Dsmall;
      }
    return g;
  };
  // the first pass's level count: the least weighted pass count, then the
  // least in-pass data movement (the stage search's cost: exchanges and
  // shuffle levels)
  const int k0max = std::min({n, dmax / 2, kcap});
  std::vector<std::pair<int, int>> groups;
  double best_cost = 1e30;
  double best_passes = 1e30;
  for (int k0 = k0max; k0 >= 1; --k0) {
    std::vector<std::pair<int, int>> g = groups_for(k0);
    const double wg = weight(g);
    if (wg > best_passes + 1e-9) continue;
    double cost = 0.0;
    bool ok = true;
    int b = 0;
    for (const auto& kd : g) {
      int D = std::min(kd.second, 2 * n);
      if (D < 2 * kd.first) D = 2 * kd.first;
      PassDesc tmp;
      double c = 0.0;
      if (!build_pass(n, b, kd.first, D, lf, cs, &tmp, nullptr, &c)) { ok = false; break; }
      cost += c;
      b += kd.first;
    }
    if (!ok) continue;
    if (wg < best_passes - 1e-9 || cost < best_cost - 1e-9) {
      best_passes = wg;
      best_cost = cost;
      groups = g;
    }
  }
  if (groups.empty()) {
    if (err) *err = "no pass plan";
    return false;
  }
  if ((int)groups.size() > kMaxQubits) {
    if (err) *err = "too many passes";
    return false;
  }
  plan->npass = (int)groups.size();
  int b = 0;
  for (int p = 0; p < plan->npass; ++p) {
    const int K = groups[p].first;
    int D = std::min(groups[p].second, 2 * n);
    if (D < 2 * K) D = 2 * K;
    if (!build_pass(n, b, K, D, lf, cs, &plan->pass[p], err)) return false;
    b += K;
  }
  for (int p = 0; p + 1 < plan->npass; ++p) set_next(&plan->pass[p], plan->pass[p + 1]);
  for (int p = 1; p < plan->npass; ++p) set_src(&plan->pass[p], plan->pass[p - 1]);
  // Occupancy: complex128 fixed-point passes convert in both directions and
  // keep two CTAs per SM (at three the 80-register budget spills).
  for (int p = 0; p < plan->npass; ++p) {
    PassDesc& pd = plan->pass[p];
    // 2^13-element complex128 tiles: a two-CTA cluster of 256 threads
    // (min_blocks 2); other 2^13 tiles: one CTA of 512 threads (1)
    // Compensated and fixed-point complex64 (127-128 registers at two CTAs per
    // SM) run faster at three: the compensated passes compiled for their tile
    // layout (tpd_shape.h) fit 80 registers without spills (n = 15: 14.90 ->
    // 13.17 ms, n = 14: 3.31 -> 2.88 ms against two CTAs in the passes made
    // only of two-level in-register stages); the fixed-point ones keep two on
    // 2^11-element tiles only (n = 15 pass 3: 8.00 -> 7.68 ms; on 2^12 tiles,
    // n = 14 passes 2-3, three wins: 1.85 / 1.60 against 2.23 / 1.98 ms).
    bool pairs_only = pd.nstage > 1;
    for (int s = 0; s < pd.nstage; ++s)
      if (pd.st[s].npair != 2 || pd.st[s].nshfl != 0) pairs_only = false;
    const bool two_c64 = pairs_only && precision == 3 && pd.D < 12;
    const bool three = dtype == 1 && precision >= 2 && !two_c64;
    pd.min_blocks = pd.D > 12 ? (dtype == 0 ? 2 : 1) : (three ? kOccHigh : kOccLow);
  }
  return true;
}

std::string describe_plan(const Plan& plan) {
  std::string s;
  char buf[512];
  if (plan.npass == 0) {
    std::snprintf(buf, sizeof(buf), "n=%d whole-matrix kernel (%d elements in shared memory)\n", plan.n,
                  1 << (2 * plan.n));
    return buf;
  }
  for (int p = 0; p < plan.npass; ++p) {
    const PassDesc& pd = plan.pass[p];
    std::snprintf(buf, sizeof(buf), "pass %d: levels [%d,%d) D=%d tiles=%lld ctas=%d gbits=", p, pd.b,
                  pd.b + pd.K, pd.D, (long long)pd.ntiles, pd.min_blocks);
    s += buf;
    for (int i = 0; i < pd.D; ++i) {
      std::snprintf(buf, sizeof(buf), "%s%d", i ? "," : "", pd.gbit[i]);
      s += buf;
    }
    s += " cls=";
    for (int i = 0; i < pd.D; ++i) {
      std::snprintf(buf, sizeof(buf), "%s%d", i ? "," : "", pd.cls_w[i]);
      s += buf;
    }
    // the compiled tile layout (tpd_shape.h) this pass's layout equals, or -1
    std::snprintf(buf, sizeof(buf), " shape=%d", match_shape(pd));
    s += buf;
    for (int si = 0; si < pd.nstage; ++si) {
      const Stage& st = pd.st[si];
      std::snprintf(buf, sizeof(buf), " | stage %d: pairs=%d shfl=%d reg=", si, st.npair, st.nshfl);
      s += buf;
      for (int i = 0; i < kRegBits; ++i) {
        std::snprintf(buf, sizeof(buf), "%s%d", i ? "," : "", st.reg[i]);
        s += buf;
      }
      std::snprintf(buf, sizeof(buf), " lane=%d,%d,%d,%d,%d", st.lane[0], st.lane[1], st.lane[2], st.lane[3],
                    st.lane[4]);
      s += buf;
      s += " warp=";
      for (int i = 0; i < pd.D - kMinTileBits; ++i) {
        std::snprintf(buf, sizeof(buf), "%s%d", i ? "," : "", st.warp[i]);
        s += buf;
      }
      s += " shfl_lane=";
      for (int i = 0; i < st.nshfl; ++i) {
        std::snprintf(buf, sizeof(buf), "%s%d", i ? "," : "", st.shfl_lane[i]);
        s += buf;
      }
    }
    s += "\n";
  }
  return s;
}

}  // namespace tpd
