// MIS-2 aggregation (internal).
#pragma once

#include "common.cuh"

namespace saamg {

// Device scratch of the aggregation: n bytes x2, 8n bytes, 3 n ints and one counter.
struct AggScratch {
  unsigned char* state;
  unsigned char* o1;
  unsigned long long* m1;
  int* counter;   // 2 ints
  int* root1;
  int* aggroot;
  int* rank;
  int* list = nullptr;  // n ints for the late MIS-2 rounds (NULL: every round visits all rows)
};

struct AggScratchBufs {
  Buf<unsigned char> state, o1;
  Buf<unsigned long long> m1;
  Buf<int> counter, root1, aggroot, rank;
  void alloc(int n, cudaStream_t s);
  AggScratch view() const;
};

// Root flags and aggregate index (roots numbered by ascending row) of the graph given by
// the CSR pattern (rowptr, col); ids = node ids (NULL: the row index).  Returns the number
// of aggregates.  Synchronises the stream once per round.
int mis2_aggregate(int n, const int* rowptr, const int* col, long long nnz, const unsigned* ids,
                   uint32_t seed, unsigned char* root, int* agg, const AggScratch& w,
                   cudaStream_t s);

// Level-0 graph: the 7-point star on the line structure, i.e. the pattern of the assembled
// level-0 matrix (neighbour q of a row exists when bit q of nbmask is set; order -x, +x, -y,
// +y, -z, +z).  Node ids are the box indices i + nx (j + ny k).
struct GridGraph {
  const LineInfo* lines;
  const int4* nbr;      // row offsets to the -y, +y, -z, +z lines
  const int2* chunks;   // (line, offset) of <= 32 consecutive rows
  int nchunks;
  const unsigned char* nbmask;
  unsigned nx, nxy;     // id strides in y and z
  const int* rline;     // line of every row (the list rounds start from a row)
};

// mis2_aggregate on the level-0 graph, walking the line structure instead of a CSR pattern;
// the same rounds, priorities and phases, so the same roots and aggregates.
int mis2_aggregate_grid(int n, const GridGraph& g, const unsigned* ids, uint32_t seed,
                        unsigned char* root, int* agg, const AggScratch& w, cudaStream_t s);

// The paper's own aggregation (Sec. 3.2): the cubes of 3 x 3 x 3 lattice nodes.  Node v has
// the lattice id ids[v] = i + d0 (j + d1 k) on the dims lattice; every cube holding a node
// is an aggregate, numbered by ascending cube index; root = the aggregate's smallest row.
// next_ids (allocated here) receives each aggregate's cube index and next_dims the cube
// lattice (ceil(d / 3) per axis).  Returns the number of aggregates.
int cube_aggregate(int n, const unsigned* ids, const int dims[3], int* agg, unsigned char* root,
                   Buf<unsigned>& next_ids, int next_dims[3], cudaStream_t s);

// The same aggregation with every temporary in caller-provided scratch (w and `tiles`,
// scan_u8_tiles_needed(n) entries); allocates nothing.
int mis2_aggregate_into(int n, const int* rowptr, const int* col, long long nnz,
                        const unsigned* ids, uint32_t seed, unsigned char* root, int* agg,
                        const AggScratch& w, long long* tiles, cudaStream_t s);

}  // namespace saamg
