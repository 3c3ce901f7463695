// layout.h -- host-side layout of a plan's rows (no device code).
//
// Lanes per row, the streaming path's row classes, the bank-balanced entry
// order within a row, the lane-interleaved order of the streaming path and the
// cutting of row lists into the row-pass chunks.  Used at plan creation, and
// compiled on its own by the CPU tests that check these functions.
#pragma once

#include <stdint.h>
#include <vector_types.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <exception>
#include <thread>
#include <vector>

#include "chunk.h"

namespace rpt {
namespace layout {

// Runs body(i, t) for every i in [0, count) on min(nt, count) threads, t being
// the thread's index (the calling thread is thread 0); items are taken one after
// another.  An exception in a thread (out of memory) stops the others from
// taking new items and is rethrown here once every thread has joined.
template <typename F>
inline void parallel_for(int count, int nt, F&& body) {
  const int t_n = std::max(1, std::min(nt, count));
  std::atomic<int> next(0);
  std::atomic<bool> failed(false);
  std::vector<std::exception_ptr> err(t_n);
  auto loop = [&](int t) {
    try {
      for (int i = next++; i < count && !failed; i = next++) body(i, t);
    } catch (...) {
      err[t] = std::current_exception();
      failed = true;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < t_n; ++t) th.emplace_back(loop, t);
  loop(0);
  for (auto& t : th) t.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

// Lanes per row: the smallest power of two G >= min_lanes with G * kKeep >= len
// (at most 32).  min_lanes > 1 keeps the rows that share one warp instruction few:
// lanes of different rows can hit the same spot column in the same shared-memory
// atomic, which serialises; short rows (the dose periphery) often do.
constexpr int kKeep = 8;   // entries per lane held in registers by the row-pass kernels
inline int lanes_for(int len, int min_lanes, int keep = kKeep) {
  int g = min_lanes;
  while (g < 32 && g * keep < len) g <<= 1;
  return g;
}

// Per-scenario row lists (non-empty rows only, sorted by decreasing length):
// rec_base[s] .. rec_base[s] + nrows[s] are the rows of scenario s, followed by
// a terminator record holding the scenario's entry count.
struct RowLists {
  std::vector<int> rec_base;   // [N+1]
  std::vector<int> nrows;      // [N]
  std::vector<int4> rec;       // {start, c_s w, p, kept-row index}
};

inline double row_cost(int len, double per_lane, int min_lanes) {
  return (double)len + per_lane * lanes_for(len, min_lanes);
}

// Row-length classes of the streaming path (see k_rowpass_stream): lanes per row
// 8/16/32/32/32 for padded rows of at most 32/64/128/256/any entries.
inline int stream_class(int len) {
  const int q = (len + 3) >> 2;   // quads of the padded row
  return q <= 8 ? 0 : q <= 16 ? 1 : q <= 32 ? 2 : q <= 64 ? 3 : 4;
}
constexpr int kStreamLanes[5] = {8, 16, 32, 32, 32};
inline int stream_lanes(int len) { return kStreamLanes[stream_class(len)]; }

// Cut every scenario's row list into chunks of rows of one class (lanes per row
// for the ring, the streaming class otherwise), at most cmax entries in the
// 16-entry aligned span and rmax rows.  scen_chunk[s]..scen_chunk[s+1] are
// scenario s's chunks.  For the ring, returns false if a single row does not fit
// a stage; the streaming path takes such a row as a chunk of its own.
inline bool build_chunks(const RowLists& R, const std::vector<int64_t>& base, int N, int cmax, int rmax, bool stream,
                         int min_lanes, std::vector<ChunkDesc>* chunks, std::vector<int>* scen_chunk,
                         int keep = kKeep) {
  scen_chunk->assign(N + 1, 0);
  auto cls = [&](int len) { return stream ? stream_class(len) : lanes_for(len, min_lanes, keep); };
  for (int s = 0; s < N; ++s) {
    (*scen_chunk)[s] = (int)chunks->size();
    const int4* r = &R.rec[R.rec_base[s]];
    int q = 0;
    while (q < R.nrows[s]) {
      const int g0 = cls(r[q + 1].x - r[q].x);
      const int64_t g_al = (base[s] + r[q].x) & ~(int64_t)15;
      int qe = q;
      while (qe < R.nrows[s] && qe - q < rmax && cls(r[qe + 1].x - r[qe].x) == g0) {
        const int64_t g_end = (base[s] + r[qe + 1].x + 15) & ~(int64_t)15;
        if (g_end - g_al > cmax && !(stream && qe == q)) break;
        ++qe;
      }
      if (qe == q) return false;
      const int64_t n_ent = std::max<int64_t>(16, ((base[s] + r[qe].x + 15) & ~(int64_t)15) - g_al);
      if (n_ent > (int64_t)1 << 28) return false;
      ChunkDesc ch{};
      ch.g_al = g_al;
      ch.row_begin = q;
      ch.n_rows = qe - q;
      ch.n_ent = (int)n_ent;
      ch.group = stream ? kStreamLanes[g0] : g0;
      ch.s = s;
      ch.pad = stream ? g0 : 0;
      chunks->push_back(ch);
      q = qe;
    }
  }
  (*scen_chunk)[N] = (int)chunks->size();
  return true;
}

// Reorder a row's entries (the order is free: a pass sums over them) so that
// every aligned group of G consecutive entries, the entries that the G lanes of
// the row touch in one instruction, falls in as many distinct shared-memory banks
// (spot column mod 32) as the row allows: each group takes one entry from each of
// the banks with the most entries left, largest first.  The gather from v_s and
// the scatter into the accumulator then conflict less.
struct BankScratch {
  std::vector<int> order, idx;
  std::vector<int32_t> c;
  std::vector<float> v;
};

inline void bank_order(const int32_t* col, int len, int G, BankScratch& S) {
  int cnt[32] = {0}, start[33], cur[32];
  for (int i = 0; i < len; ++i) ++cnt[col[i] & 31];
  start[0] = 0;
  for (int b = 0; b < 32; ++b) start[b + 1] = start[b] + cnt[b];
  S.order.clear();
  if (len <= 0) return;
  S.idx.resize(len);
  S.order.resize(len);
  for (int b = 0; b < 32; ++b) cur[b] = start[b];
  for (int i = 0; i < len; ++i) S.idx[cur[col[i] & 31]++] = i;   // entries by bank, stable
  for (int b = 0; b < 32; ++b) cur[b] = start[b];
  // non-empty banks by entries left, largest first (ties: lower bank first),
  // kept as keys (left << 5) | (31 - bank) in decreasing order; the order
  // carries over from group to group, where it changes little, and is restored
  // by insertion sort after the emptied banks are dropped
  int key[32], nb = 0;
  for (int b = 0; b < 32; ++b)
    if (cnt[b] > 0) key[nb++] = (cnt[b] << 5) | (31 - b);
  int o = 0;
  while (o < len) {
    int kept = 0;
    for (int k = 0; k < nb; ++k)
      if (key[k] >= 32) key[kept++] = key[k];
    nb = kept;
    for (int k = 1; k < nb; ++k) {
      const int x = key[k];
      int m = k;
      for (; m > 0 && x > key[m - 1]; --m) key[m] = key[m - 1];
      key[m] = x;
    }
    const int want = std::min(G, len - o);
    int taken = 0;
    for (int k = 0; k < nb && taken < want; ++k, ++taken) {
      const int b = 31 - (key[k] & 31);
      S.order[o++] = S.idx[cur[b]++];
      key[k] -= 32;
    }
    // fewer non-empty banks than lanes: fill the group from the largest banks again
    for (int k = 0; taken < want; k = (k + 1) % nb) {
      if (key[k] >= 32) {
        const int b = 31 - (key[k] & 31);
        S.order[o++] = S.idx[cur[b]++];
        key[k] -= 32;
        ++taken;
      }
    }
  }
}

inline void bank_balance(int32_t* col, float* val, int len, int G, BankScratch& S) {
  if (len <= 1) return;
  bank_order(col, len, G, S);
  S.c.assign(col, col + len);
  S.v.assign(val, val + len);
  for (int i = 0; i < len; ++i) {
    col[i] = S.c[S.order[i]];
    val[i] = S.v[S.order[i]];
  }
}

// The streaming path reads a row as quads (4 stored entries) with lane l of the
// row's G lanes taking quads l, l + G, ...; its rows are stored lane-interleaved
// so that, for each quad block b (g_b <= G lanes) and each component k, the lanes
// hold consecutive entries of the row:
//   stored[4 (b G + l) + k] = row[4 b G + k g_b + l].
// (Row order is free: the pass sums over the row's entries.)  Consecutive
// entries have nearby spot columns, which then fall in different shared-memory
// banks for the gather and the scatter.  plen: the padded row length (a
// multiple of 4); col_out/val_out: plen entries.
inline void interleave_row(const int32_t* col, const float* val, int plen, int G, int32_t* col_out,
                           float* val_out) {
  const int nq = plen / 4;
  for (int b = 0; b * G < nq; ++b) {
    const int gb = std::min(G, nq - b * G);
    for (int l = 0; l < gb; ++l)
      for (int k = 0; k < 4; ++k) {
        const int dst = 4 * (b * G + l) + k;
        const int src = 4 * b * G + k * gb + l;
        col_out[dst] = col[src];
        val_out[dst] = val[src];
      }
  }
}


// ---- row bundles (the bundled ring path) -------------------------------------
// A scenario's non-empty rows, in the plan's kept-row order (neighbouring voxels
// when the caller numbers voxels spatially), are grouped kBunRows at a time.
// A bundle stores the sorted union of its rows' spot columns once, and for each
// such "block column" the kBunRows values of its rows (zero where a row has no
// entry there).  One index then serves several entries, and the row pass does
// one gather from the spot vector and one scatter into the accumulator per
// block column instead of one per entry.  The block columns of a bundle are
// bank-balanced for the bundle's lanes; bundles are sorted by decreasing
// block-column count so that chunks hold bundles of one lane class.
constexpr int kBunRows = kBundleRows;   // rows per bundle
constexpr int kBunKeep = kBundleKeep;   // block columns per lane held in registers by the bundled kernel
constexpr int kBunMinLanes = 8;

inline int bundle_lanes(int ncols) { return lanes_for(ncols, kBunMinLanes, kBunKeep); }

// Input rows of one scenario (non-empty, kept order): kept index, the row's
// entries (strictly increasing columns), c_s w_i and p_i as stored.
struct BundleInRow {
  int32_t kept;
  const int32_t* col;
  const float* val;
  int32_t len;
  float wc, p;
};

// One scenario's bundles.  rec: 4 int4 per bundle, in sorted order
// {block-column offset, 0, 0, 0}, {c_s w_i of rows 0..3}, {p_i of rows 0..3},
// {kept index of rows 0..3 (-1: no row)}, then 4 int4 holding the scenario's
// block-column count.  col [nbc], val [nbc][kBunRows].  pos_of: sorted position
// of the q-th bundle in creation (kept-row) order.
struct BundleScen {
  std::vector<int4> rec;
  std::vector<int32_t> col;
  std::vector<float> val;
  std::vector<int32_t> pos_of;
  int nb = 0;
  int64_t nbc = 0;
};

inline int32_t f2i_bits(float f) {
  int32_t i;
  std::memcpy(&i, &f, 4);
  return i;
}

// Block columns of the bundle of rows r0 .. r0 + rn - 1: the union of the rows'
// columns by a kBunRows-way merge (each row's next column held as its head,
// INT32_MAX once the row is exhausted; columns are below INT32_MAX).  With C
// and V, the union's columns and their kBunRows values (zero where a row lacks
// the column) are written there; returns the union's size.
inline int merge_bundle(const std::vector<BundleInRow>& rows, int r0, int rn, int32_t* C, float* V) {
  const int32_t* col[kBunRows];
  const float* val[kBunRows];
  int len[kBunRows], pos[kBunRows];
  int32_t head[kBunRows];
  for (int r = 0; r < kBunRows; ++r) {
    const bool has = r < rn;
    col[r] = has ? rows[r0 + r].col : nullptr;
    val[r] = has ? rows[r0 + r].val : nullptr;
    len[r] = has ? rows[r0 + r].len : 0;
    pos[r] = 0;
    head[r] = len[r] > 0 ? col[r][0] : INT32_MAX;
  }
  int n = 0;
  for (;;) {
    int32_t cmin = head[0];
    for (int r = 1; r < kBunRows; ++r) cmin = std::min(cmin, head[r]);
    if (cmin == INT32_MAX) break;
    if (C) C[n] = cmin;
    for (int r = 0; r < kBunRows; ++r) {
      const bool hit = head[r] == cmin;
      if (C) V[(size_t)n * kBunRows + r] = hit ? val[r][pos[r]] : 0.f;
      if (hit) {
        ++pos[r];
        head[r] = pos[r] < len[r] ? col[r][pos[r]] : INT32_MAX;
      }
    }
    ++n;
  }
  return n;
}

// The bundling in three steps, so that the work of several scenarios can be
// spread over threads:
//   bundle_widths: the widths (block columns) of bundles q0 .. q1 - 1;
//   bundle_order:  from all widths, the sorted order (widest first, stable),
//                  pos_of, the records and the storage of out;
//   bundle_fill:   the block columns of sorted bundles k0 .. k1 - 1, each merged
//                  into scratch, bank-ordered and written once at its offset.
inline int bundle_count(const std::vector<BundleInRow>& rows) {
  return ((int)rows.size() + kBunRows - 1) / kBunRows;
}

inline void bundle_widths(const std::vector<BundleInRow>& rows, int q0, int q1, int32_t* width) {
  const int nr = (int)rows.size();
  for (int q = q0; q < q1; ++q) {
    const int r0 = q * kBunRows, rn = std::min(kBunRows, nr - r0);
    width[q] = merge_bundle(rows, r0, rn, nullptr, nullptr);
  }
}

inline void bundle_order(const std::vector<BundleInRow>& rows, const std::vector<int32_t>& width, BundleScen* out,
                         std::vector<int>* ord) {
  const int nr = (int)rows.size();
  const int nb = (int)width.size();
  ord->resize(nb);
  for (int q = 0; q < nb; ++q) (*ord)[q] = q;
  std::stable_sort(ord->begin(), ord->end(), [&](int a, int b) { return width[a] > width[b]; });
  out->nb = nb;
  out->pos_of.assign(nb, 0);
  out->rec.assign((size_t)4 * (nb + 1), int4{0, 0, 0, 0});
  int64_t off = 0;
  for (int k = 0; k < nb; ++k) {
    const int q = (*ord)[k];
    out->pos_of[q] = k;
    const int r0 = q * kBunRows, rn = std::min(kBunRows, nr - r0);
    int4* R4 = &out->rec[(size_t)4 * k];
    R4[0] = int4{(int)off, 0, 0, 0};
    int wc[kBunRows] = {0}, pp[kBunRows] = {0}, kp[kBunRows] = {-1, -1, -1, -1};
    for (int r = 0; r < rn; ++r) {
      wc[r] = f2i_bits(rows[r0 + r].wc);
      pp[r] = f2i_bits(rows[r0 + r].p);
      kp[r] = rows[r0 + r].kept;
    }
    R4[1] = int4{wc[0], wc[1], wc[2], wc[3]};
    R4[2] = int4{pp[0], pp[1], pp[2], pp[3]};
    R4[3] = int4{kp[0], kp[1], kp[2], kp[3]};
    off += width[q];
  }
  out->rec[(size_t)4 * nb] = int4{(int)off, 0, 0, 0};
  out->nbc = off;
  out->col.resize((size_t)off);
  out->val.resize((size_t)off * kBunRows);
}

inline void bundle_fill(const std::vector<BundleInRow>& rows, const std::vector<int32_t>& width,
                        const std::vector<int>& ord, int k0, int k1, BundleScen* out, BankScratch& S) {
  const int nr = (int)rows.size();
  int wmax = 0;
  for (int k = k0; k < k1; ++k) wmax = std::max(wmax, width[ord[k]]);
  if ((int)S.c.size() < wmax) S.c.resize((size_t)wmax);
  if (S.v.size() < (size_t)wmax * kBunRows) S.v.resize((size_t)wmax * kBunRows);
  for (int k = k0; k < k1; ++k) {
    const int q = ord[k];
    const int r0 = q * kBunRows, rn = std::min(kBunRows, nr - r0);
    const int64_t off = out->rec[(size_t)4 * k].x;
    const int len = merge_bundle(rows, r0, rn, S.c.data(), S.v.data());
    int32_t* oc = out->col.data() + off;
    float* ov = out->val.data() + off * kBunRows;
    if (len > 1) {
      // bank-balanced block-column order for the bundle's lanes
      bank_order(S.c.data(), len, bundle_lanes(len), S);
      for (int i = 0; i < len; ++i) {
        const int src = S.order[i];
        oc[i] = S.c[src];
        for (int r = 0; r < kBunRows; ++r) ov[(size_t)i * kBunRows + r] = S.v[(size_t)src * kBunRows + r];
      }
    } else if (len == 1) {
      oc[0] = S.c[0];
      for (int r = 0; r < kBunRows; ++r) ov[r] = S.v[r];
    }
  }
}

// One scenario's bundles on the calling thread.
inline void build_bundles(const std::vector<BundleInRow>& rows, BundleScen* out, BankScratch& S) {
  const int nb = bundle_count(rows);
  std::vector<int32_t> width(nb);
  bundle_widths(rows, 0, nb, width.data());
  std::vector<int> ord;
  bundle_order(rows, width, out, &ord);
  bundle_fill(rows, width, ord, 0, nb, out, S);
}

// Every scenario's bundles, the same as build_bundles per scenario, with the
// widths and the fills of all scenarios cut into ranges of kBunRange bundles
// that nt threads take one after another (the order step runs per scenario).
// An exception in a thread is rethrown on the caller's.
constexpr int kBunRange = 2048;

inline void build_bundles_all(const std::vector<std::vector<BundleInRow>>& rows, std::vector<BundleScen>* out,
                              int nt) {
  const int N = (int)rows.size();
  out->assign(N, BundleScen());
  std::vector<std::vector<int32_t>> width(N);
  std::vector<std::vector<int>> ord(N);
  std::vector<int2> items;   // (scenario, first bundle) of every range
  for (int s = 0; s < N; ++s) {
    width[s].resize(bundle_count(rows[s]));
    for (int q = 0; q < (int)width[s].size(); q += kBunRange) items.push_back(int2{s, q});
  }
  std::vector<BankScratch> scratch(std::max(1, std::min(nt, (int)items.size())));
  parallel_for((int)items.size(), nt, [&](int i, int) {
    const int s = items[i].x, q0 = items[i].y;
    bundle_widths(rows[s], q0, std::min(q0 + kBunRange, (int)width[s].size()), width[s].data());
  });
  parallel_for(N, nt, [&](int s, int) { bundle_order(rows[s], width[s], &(*out)[s], &ord[s]); });
  parallel_for((int)items.size(), (int)scratch.size(), [&](int i, int t) {
    const int s = items[i].x, k0 = items[i].y;
    bundle_fill(rows[s], width[s], ord[s], k0, std::min(k0 + kBunRange, (int)width[s].size()), &(*out)[s],
                scratch[t]);
  });
}

}  // namespace layout
}  // namespace rpt
