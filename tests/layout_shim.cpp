// C entry points over the plan-layout header, built by tests/test_layout_host.py
// with the host compiler alone (no CUDA runtime, no device), so that the host
// layout logic of plan creation is tested on the CPU.
#include <cstdint>
#include <cstring>
#include <vector>

#include "layout.h"

using namespace rpt;
using namespace rpt::layout;

extern "C" {

int shim_lanes_for(int len, int min_lanes) { return lanes_for(len, min_lanes); }
int shim_stream_class(int len) { return stream_class(len); }
int shim_stream_lanes(int len) { return stream_lanes(len); }

void shim_bank_balance(int32_t* col, float* val, int len, int G) {
  BankScratch S;
  bank_balance(col, val, len, G, S);
}

void shim_interleave_row(const int32_t* col, const float* val, int plen, int G, int32_t* col_out,
                         float* val_out) {
  interleave_row(col, val, plen, G, col_out, val_out);
}

// Row lists from padded row lengths (scenario-major, nrows[s] rows each, in
// list order); base[s] = the scenario's first stored entry.  Writes up to cap
// chunks (fields in separate arrays) and scen_chunk[N+1]; returns the chunk
// count, -1 when build_chunks refuses, -2 when cap is too small.
int shim_build_chunks(int N, const int* nrows, const int* plen, const int64_t* base, int cmax, int rmax,
                      int stream, int min_lanes, int cap, int64_t* g_al, int* row_begin, int* n_rows,
                      int* n_ent, int* group, int* s_out, int* pad, int* scen_chunk) {
  RowLists R;
  R.rec_base.assign(N + 1, 0);
  R.nrows.assign(nrows, nrows + N);
  for (int s = 0; s < N; ++s) R.rec_base[s + 1] = R.rec_base[s] + nrows[s] + 1;
  R.rec.resize(R.rec_base[N]);
  int k = 0;
  for (int s = 0; s < N; ++s) {
    int pos = 0;
    for (int q = 0; q < nrows[s]; ++q) {
      R.rec[R.rec_base[s] + q] = int4{pos, 0, 0, q};
      pos += plen[k++];
    }
    R.rec[R.rec_base[s] + nrows[s]] = int4{pos, 0, 0, 0};
  }
  std::vector<int64_t> b(base, base + N);
  std::vector<ChunkDesc> chunks;
  std::vector<int> sc;
  if (!build_chunks(R, b, N, cmax, rmax, stream != 0, min_lanes, &chunks, &sc)) return -1;
  if ((int)chunks.size() > cap) return -2;
  for (size_t i = 0; i < chunks.size(); ++i) {
    g_al[i] = chunks[i].g_al;
    row_begin[i] = chunks[i].row_begin;
    n_rows[i] = chunks[i].n_rows;
    n_ent[i] = chunks[i].n_ent;
    group[i] = chunks[i].group;
    s_out[i] = chunks[i].s;
    pad[i] = chunks[i].pad;
  }
  for (int s = 0; s <= N; ++s) scen_chunk[s] = sc[s];
  return (int)chunks.size();
}

// Bundles of one scenario's rows (CSR rp [nrows+1], ci, va; row i has kept
// index kept[i], weight wc[i] and prescription pr[i]).  Returns the block-column
// count (or -2 when cap_bc / cap_b is too small) and writes col [nbc], val
// [nbc][4], rec [(nb+1)*4][4] (int32 fields), pos_of [nb], *nb_out.
int64_t shim_build_bundles(int nrows, const int32_t* rp, const int32_t* ci, const float* va, const int32_t* kept,
                           const float* wc, const float* pr, int64_t cap_bc, int cap_b, int32_t* col, float* val,
                           int32_t* rec, int32_t* pos_of, int* nb_out) {
  std::vector<BundleInRow> rows(nrows);
  for (int i = 0; i < nrows; ++i)
    rows[i] = BundleInRow{kept[i], ci + rp[i], va + rp[i], rp[i + 1] - rp[i], wc[i], pr[i]};
  BundleScen B;
  BankScratch S;
  build_bundles(rows, &B, S);
  *nb_out = B.nb;
  if (B.nbc > cap_bc || B.nb > cap_b) return -2;
  for (int64_t k = 0; k < B.nbc; ++k) {
    col[k] = B.col[k];
    for (int r = 0; r < kBunRows; ++r) val[k * kBunRows + r] = B.val[k * kBunRows + r];
  }
  for (size_t k = 0; k < B.rec.size(); ++k) {
    rec[4 * k] = B.rec[k].x;
    rec[4 * k + 1] = B.rec[k].y;
    rec[4 * k + 2] = B.rec[k].z;
    rec[4 * k + 3] = B.rec[k].w;
  }
  for (int q = 0; q < B.nb; ++q) pos_of[q] = B.pos_of[q];
  return B.nbc;
}

int shim_bundle_lanes(int ncols) { return bundle_lanes(ncols); }

// The bundles of N scenarios (CSR each) by the threaded driver with nt threads,
// compared with build_bundles scenario by scenario: 1 if every array is equal.
int shim_bundles_all_equal(int N, const int* nrows, const int32_t* const* rp, const int32_t* const* ci,
                           const float* const* va, int nt) {
  std::vector<std::vector<BundleInRow>> rows(N);
  for (int s = 0; s < N; ++s) {
    rows[s].resize(nrows[s]);
    for (int i = 0; i < nrows[s]; ++i)
      rows[s][i] = BundleInRow{5 * i + s, ci[s] + rp[s][i], va[s] + rp[s][i], rp[s][i + 1] - rp[s][i], 0.25f * i,
                               1.0f + s};
  }
  std::vector<BundleScen> A;
  build_bundles_all(rows, &A, nt);
  if ((int)A.size() != N) return 0;
  BankScratch S;
  for (int s = 0; s < N; ++s) {
    BundleScen B;
    build_bundles(rows[s], &B, S);
    if (A[s].nb != B.nb || A[s].nbc != B.nbc || A[s].col != B.col || A[s].val != B.val || A[s].pos_of != B.pos_of ||
        A[s].rec.size() != B.rec.size())
      return 0;
    for (size_t k = 0; k < B.rec.size(); ++k)
      if (std::memcmp(&A[s].rec[k], &B.rec[k], sizeof(int4)) != 0) return 0;
  }
  return 1;
}

}  // extern "C"
