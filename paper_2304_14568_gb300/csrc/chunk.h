// chunk.h -- the row-pass work unit, shared by the host layout code and the kernels.
#pragma once

namespace rpt {

// Row bundles (bundled ring path): rows per bundle, and block columns per lane
// that the bundled kernel keeps in registers (the lane classes of the chunks
// are cut for it).
constexpr int kBundleRows = 4;
constexpr int kBundleKeep = 6;

// A run of consecutive rows of one scenario's row list, of one lanes-per-row
// class, copied to shared memory (ring path) or claimed by a warp (streaming
// path) as a unit.
struct ChunkDesc {
  long long g_al;                     // first copied entry (global index, multiple of 16)
  int row_begin;                      // first row of the chunk (index in the scenario's row list)
  int n_rows;                         // rows in the chunk (-1: end-of-work marker)
  int n_ent;                          // copied entries (multiple of 16)
  int group;                          // lanes per row (1..32), the same for every row of the chunk
  int s;                              // scenario
  int pad;                            // streaming path: row-length class of the chunk's rows
};

}  // namespace rpt
