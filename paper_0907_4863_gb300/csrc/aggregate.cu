// Aggregation for the tentative prolongator (Sec. 3.2, "Prolongation operator"):
// aggregates seeded by a deterministic distance-2 maximal independent set (MIS-2) of the
// adjacency graph G_l of A_l, computed in synchronous rounds.
//
// Priority of node v: (fmix32(id_v ^ seed), v) compared lexicographically.  Rows are
// numbered in ascending id, so this is the same order as (fmix32(id ^ seed), id).
// Round: an undecided node joins when its priority is the largest among the undecided
// nodes within graph distance 2; afterwards every undecided node within distance 2 of a
// member leaves.  With fixed priorities these rounds select exactly the set of the
// sequential greedy rule (visit by decreasing priority, join unless a member is within
// distance 2) -- the determinism result for parallel greedy MIS of Blelloch, Fineman and
// Shun (2012), applied to the square of the graph.
#include <mutex>

#include "aggregate.cuh"

namespace saamg {

namespace {

// MurmurHash3 32-bit finaliser (public domain): xor-shift 16, multiply 0x85ebca6b,
// xor-shift 13, multiply 0xc2b2ae35, xor-shift 16.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ unsigned long long prio(const unsigned* ids, int row, uint32_t seed) {
  uint32_t id = ids ? ids[row] : (uint32_t)row;
  // +1 keeps 0 free as "no candidate"; rows < 2^31 so this never wraps
  return (((unsigned long long)fmix32(id ^ seed) << 32) | (unsigned long long)(uint32_t)row) + 1ull;
}

template <class T>
__device__ __forceinline__ T group_max(T v, int G) {
  for (int o = G / 2; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o, G);
    v = w > v ? w : v;
  }
  return v;
}

__device__ __forceinline__ int group_or(int v, int G) {
  for (int o = G / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Loop shared by the kernels below: 32/G rows per warp, uniform trip count per warp.
#define SAAMG_ROW_LOOP(G)                                                          \
  const int lane = threadIdx.x & 31;                                               \
  const int gl = lane % (G);                                                       \
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;                   \
  const int nwarps = (gridDim.x * blockDim.x) >> 5;                                \
  for (int wbase = warp * (32 / (G)); wbase < n; wbase += nwarps * (32 / (G)))

// m1[j] = max priority of the undecided nodes in N[j] (0 if none)
template <int G>
__global__ void mis_max1_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const unsigned char* __restrict__ state, const unsigned* __restrict__ ids,
                           uint32_t seed, unsigned long long* __restrict__ m1) {
  SAAMG_ROW_LOOP(G) {
    int row = wbase + lane / G;
    unsigned long long acc = 0;
    if (row < n && gl == 0 && state[row] == 0) acc = prio(ids, row, seed);  // closed N[j]
    if (row < n)
      for (int p = rowptr[row] + gl; p < rowptr[row + 1]; p += G) {
        int u = col[p];
        if (state[u] == 0) {
          unsigned long long k = prio(ids, u, seed);
          acc = k > acc ? k : acc;
        }
      }
    acc = group_max(acc, G);
    if (row < n && gl == 0) m1[row] = acc;
  }
}

// an undecided node whose priority is the maximum over N[N[i]] joins
template <int G>
__global__ void mis_max2_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           unsigned char* __restrict__ state, const unsigned* __restrict__ ids,
                           uint32_t seed, const unsigned long long* __restrict__ m1) {
  SAAMG_ROW_LOOP(G) {
    int row = wbase + lane / G;
    bool und = row < n && state[row] == 0;
    unsigned long long acc = (und && gl == 0) ? m1[row] : 0ull;
    if (und)
      for (int p = rowptr[row] + gl; p < rowptr[row + 1]; p += G) {
        unsigned long long k = m1[col[p]];
        acc = k > acc ? k : acc;
      }
    acc = group_max(acc, G);
    if (und && gl == 0 && acc == prio(ids, row, seed)) state[row] = 1;
  }
}

// o1[j] = 1 if N[j] holds a member
template <int G>
__global__ void mis_or1_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const unsigned char* __restrict__ state, unsigned char* __restrict__ o1) {
  SAAMG_ROW_LOOP(G) {
    int row = wbase + lane / G;
    int any = (row < n && gl == 0) ? (state[row] == 1) : 0;
    if (row < n)
      for (int p = rowptr[row] + gl; p < rowptr[row + 1]; p += G) any |= (state[col[p]] == 1);
    any = group_or(any, G);
    if (row < n && gl == 0) o1[row] = (unsigned char)any;
  }
}

// undecided nodes within distance 2 of a member leave; count the rest
template <int G>
__global__ void mis_or2_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                          unsigned char* __restrict__ state, const unsigned char* __restrict__ o1,
                          int* __restrict__ undecided) {
  int cnt = 0;
  SAAMG_ROW_LOOP(G) {
    int row = wbase + lane / G;
    bool und = row < n && state[row] == 0;
    int any = (und && gl == 0) ? o1[row] : 0;
    if (und)
      for (int p = rowptr[row] + gl; p < rowptr[row + 1]; p += G) any |= o1[col[p]];
    any = group_or(any, G);
    if (und && gl == 0) {
      if (any) state[row] = 2;
      else ++cnt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(undecided, cnt);
}

// --- late rounds on a list of the undecided rows ---------------------------------------
// Once few rows are undecided, a round visits only them: the join test looks at the closed
// distance-2 neighbourhood of a listed row directly (the same set max1 / max2 cover), joins
// are applied after every test has read the snapshot, and then the listed rows with a member
// within distance 2 leave.  The list order does not matter: every decision reads the same
// state.

__global__ void mis_list_k(int n, const unsigned char* __restrict__ state, int* __restrict__ list,
                           int* __restrict__ nlist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool und = i < n && state[i] == 0;
  const unsigned m = __ballot_sync(0xffffffffu, und);
  if (!m) return;  // the whole warp
  int base = 0;
  if (lane == 0) base = atomicAdd(nlist, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (und) list[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// join[i] = 1 if the priority of listed row i is the largest over the undecided rows within
// distance 2 (G lanes per row split the closed neighbourhood N[i]; each lane walks N[j]).
template <int G>
__global__ void mis_join_list_k(const int* __restrict__ list, const int* __restrict__ nlist,
                                const int* __restrict__ rowptr, const int* __restrict__ col,
                                const unsigned char* __restrict__ state,
                                const unsigned* __restrict__ ids, uint32_t seed,
                                unsigned char* __restrict__ join) {
  const int n = *nlist;
  SAAMG_ROW_LOOP(G) {
    const int t = wbase + lane / G;
    const bool ok = t < n;
    const int i = ok ? list[t] : 0;
    unsigned long long acc = 0;
    if (ok) {
      const int p0 = rowptr[i], p1 = rowptr[i + 1];
      for (int p = p0 - 1 + gl; p < p1; p += G) {  // p0 - 1 stands for i itself
        const int j = p < p0 ? i : col[p];
        if (state[j] == 0) {
          const unsigned long long k = prio(ids, j, seed);
          acc = k > acc ? k : acc;
        }
        for (int q = rowptr[j]; q < rowptr[j + 1]; ++q) {
          const int u = col[q];
          if (state[u] == 0) {
            const unsigned long long k = prio(ids, u, seed);
            acc = k > acc ? k : acc;
          }
        }
      }
    }
    acc = group_max(acc, G);
    if (ok && gl == 0) join[i] = acc == prio(ids, i, seed) ? 1 : 0;
  }
}

__global__ void mis_set_list_k(const int* __restrict__ list, const int* __restrict__ nlist,
                               const unsigned char* __restrict__ join,
                               unsigned char* __restrict__ state) {
  const int n = *nlist;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i = list[t];
    if (join[i]) state[i] = 1;
  }
}

// listed rows still undecided leave when a member lies within distance 2; count the rest
template <int G>
__global__ void mis_leave_list_k(const int* __restrict__ list, const int* __restrict__ nlist,
                                 const int* __restrict__ rowptr, const int* __restrict__ col,
                                 unsigned char* __restrict__ state, int* __restrict__ undecided) {
  const int n = *nlist;
  int cnt = 0;
  SAAMG_ROW_LOOP(G) {
    const int t = wbase + lane / G;
    const bool ok = t < n;
    const int i = ok ? list[t] : 0;
    const bool und = ok && state[i] == 0;
    int any = 0;
    if (und) {
      const int p0 = rowptr[i], p1 = rowptr[i + 1];
      for (int p = p0 - 1 + gl; p < p1 && !any; p += G) {
        const int j = p < p0 ? i : col[p];
        any |= state[j] == 1;
        for (int q = rowptr[j]; q < rowptr[j + 1] && !any; ++q) any |= state[col[q]] == 1;
      }
    }
    any = group_or(any, G);
    if (und && gl == 0) {
      if (any) state[i] = 2;
      else ++cnt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(undecided, cnt);
}

__global__ void roots_from_state_k(int n, const unsigned char* __restrict__ state,
                                   unsigned char* __restrict__ root) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) root[i] = state[i] == 1;
}

// phase 1: a root claims itself and its neighbours (disjoint for distinct roots)
__global__ void agg_phase1_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const unsigned char* __restrict__ root, int* __restrict__ root1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !root[i]) return;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) root1[col[p]] = i;
  root1[i] = i;
}

// phase 2: other nodes join the phase-1 aggregate whose root has the largest priority
template <int G>
__global__ void agg_phase2_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const unsigned* __restrict__ ids, uint32_t seed,
                             const int* __restrict__ root1, int* __restrict__ aggroot,
                             int* __restrict__ err) {
  SAAMG_ROW_LOOP(G) {
    int row = wbase + lane / G;
    bool need = row < n && root1[row] < 0;
    unsigned long long best = 0;
    if (need)
      for (int p = rowptr[row] + gl; p < rowptr[row + 1]; p += G) {
        int r = root1[col[p]];
        if (r >= 0) {
          unsigned long long k = prio(ids, r, seed);
          best = k > best ? k : best;
        }
      }
    best = group_max(best, G);
    if (row < n && gl == 0) {
      if (!need) {
        aggroot[row] = root1[row];
      } else if (best == 0) {
        aggroot[row] = -1;
        atomicOr(err, 1);
      } else {
        aggroot[row] = (int)(uint32_t)((best - 1ull) & 0xffffffffull);
      }
    }
  }
}

__global__ void agg_number_k(int n, const int* __restrict__ aggroot, const int* __restrict__ rank,
                             int* __restrict__ agg) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) agg[i] = aggroot[i] >= 0 ? rank[aggroot[i]] : -1;
}

// --- level 0 on the line structure ------------------------------------------
// Lane per row of a chunk; the six neighbours are row + off[q] with box ids id + dq[q].
struct Nb0 {
  int row;
  unsigned id, mask;
  int off[6];
};

__device__ __forceinline__ bool grid_row(const GridGraph& g, int c, int lane, Nb0& r) {
  const int2 ch = g.chunks[c];
  const LineInfo me = g.lines[ch.x];
  const int i = me.lo + ch.y + lane;
  if (i > me.hi) return false;
  const int4 nb = g.nbr[ch.x];
  r.row = me.start + ch.y + lane;
  r.id = (unsigned)i + g.nx * (unsigned)ch.x;
  r.mask = g.nbmask[r.row];
  r.off[0] = -1;
  r.off[1] = 1;
  r.off[2] = nb.x;
  r.off[3] = nb.y;
  r.off[4] = nb.z;
  r.off[5] = nb.w;
  return true;
}

__device__ __forceinline__ unsigned nb_id(const GridGraph& g, unsigned id, int q) {
  switch (q) {
    case 0: return id - 1u;
    case 1: return id + 1u;
    case 2: return id - g.nx;
    case 3: return id + g.nx;
    case 4: return id - g.nxy;
    default: return id + g.nxy;
  }
}

__device__ __forceinline__ unsigned long long prio_id(unsigned id, int row, uint32_t seed) {
  return (((unsigned long long)fmix32(id ^ seed) << 32) | (unsigned long long)(uint32_t)row) + 1ull;
}

#define SAAMG_CHUNK_LOOP                                                                  \
  const int lane = threadIdx.x & 31;                                                      \
  const int nw = (gridDim.x * blockDim.x) >> 5;                                           \
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < g.nchunks; c += nw)

__global__ void __launch_bounds__(256) mis0_max1_k(GridGraph g,
                                                   const unsigned char* __restrict__ state,
                                                   uint32_t seed,
                                                   unsigned long long* __restrict__ m1) {
  SAAMG_CHUNK_LOOP {
    Nb0 r;
    if (!grid_row(g, c, lane, r)) continue;
    unsigned long long acc = state[r.row] == 0 ? prio_id(r.id, r.row, seed) : 0ull;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if ((r.mask >> q) & 1u) {
        const int u = r.row + r.off[q];
        if (state[u] == 0) {
          const unsigned long long k = prio_id(nb_id(g, r.id, q), u, seed);
          acc = k > acc ? k : acc;
        }
      }
    }
    m1[r.row] = acc;
  }
}

__global__ void __launch_bounds__(256) mis0_max2_k(GridGraph g, unsigned char* __restrict__ state,
                                                   uint32_t seed,
                                                   const unsigned long long* __restrict__ m1) {
  SAAMG_CHUNK_LOOP {
    Nb0 r;
    if (!grid_row(g, c, lane, r)) continue;
    if (state[r.row] != 0) continue;
    unsigned long long acc = m1[r.row];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if ((r.mask >> q) & 1u) {
        const unsigned long long k = m1[r.row + r.off[q]];
        acc = k > acc ? k : acc;
      }
    }
    if (acc == prio_id(r.id, r.row, seed)) state[r.row] = 1;
  }
}

__global__ void __launch_bounds__(256) mis0_or1_k(GridGraph g,
                                                  const unsigned char* __restrict__ state,
                                                  unsigned char* __restrict__ o1) {
  SAAMG_CHUNK_LOOP {
    Nb0 r;
    if (!grid_row(g, c, lane, r)) continue;
    int any = state[r.row] == 1;
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if ((r.mask >> q) & 1u) any |= state[r.row + r.off[q]] == 1;
    o1[r.row] = (unsigned char)any;
  }
}

__global__ void __launch_bounds__(256) mis0_or2_k(GridGraph g, unsigned char* __restrict__ state,
                                                  const unsigned char* __restrict__ o1,
                                                  int* __restrict__ undecided) {
  int cnt = 0;
  SAAMG_CHUNK_LOOP {
    Nb0 r;
    if (!grid_row(g, c, lane, r)) continue;
    if (state[r.row] != 0) continue;
    int any = o1[r.row];
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if ((r.mask >> q) & 1u) any |= o1[r.row + r.off[q]];
    if (any) state[r.row] = 2;
    else ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(undecided, cnt);
}

// Late rounds on the list of undecided rows, on the line structure: a thread per listed row
// walks its closed distance-2 neighbourhood directly (the set max1 / max2 and or1 / or2
// cover), so a list round decides exactly as a full round.
__device__ __forceinline__ Nb0 grid_node(const GridGraph& g, int row) {
  Nb0 r;
  const int L = g.rline[row];
  const LineInfo me = g.lines[L];
  const int4 nb = g.nbr[L];
  r.row = row;
  r.id = (unsigned)(me.lo + (row - me.start)) + g.nx * (unsigned)L;
  r.mask = g.nbmask[row];
  r.off[0] = -1;
  r.off[1] = 1;
  r.off[2] = nb.x;
  r.off[3] = nb.y;
  r.off[4] = nb.z;
  r.off[5] = nb.w;
  return r;
}

__global__ void __launch_bounds__(256) mis0_join_list_k(const int* __restrict__ list,
                                                        const int* __restrict__ nlist,
                                                        GridGraph g,
                                                        const unsigned char* __restrict__ state,
                                                        uint32_t seed,
                                                        unsigned char* __restrict__ join) {
  const int n = *nlist;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const Nb0 a = grid_node(g, list[t]);
    const unsigned long long mine = prio_id(a.id, a.row, seed);
    unsigned long long acc = state[a.row] == 0 ? mine : 0ull;
    for (int q = 0; q < 6; ++q) {
      if (!((a.mask >> q) & 1u)) continue;
      const Nb0 b = grid_node(g, a.row + a.off[q]);
      if (state[b.row] == 0) {
        const unsigned long long k = prio_id(b.id, b.row, seed);
        acc = k > acc ? k : acc;
      }
      for (int q2 = 0; q2 < 6; ++q2) {
        if (!((b.mask >> q2) & 1u)) continue;
        const int v = b.row + b.off[q2];
        if (state[v] == 0) {
          const unsigned long long k = prio_id(nb_id(g, b.id, q2), v, seed);
          acc = k > acc ? k : acc;
        }
      }
    }
    join[a.row] = acc == mine ? 1 : 0;
  }
}

// listed rows still undecided leave when a member lies within distance 2; count the rest
__global__ void __launch_bounds__(256) mis0_leave_list_k(const int* __restrict__ list,
                                                         const int* __restrict__ nlist,
                                                         GridGraph g,
                                                         unsigned char* __restrict__ state,
                                                         int* __restrict__ undecided) {
  const int n = *nlist;
  int cnt = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i = list[t];
    if (state[i] != 0) continue;
    const Nb0 a = grid_node(g, i);
    int any = 0;
    for (int q = 0; q < 6 && !any; ++q) {
      if (!((a.mask >> q) & 1u)) continue;
      const int u = i + a.off[q];
      any |= state[u] == 1;
      const Nb0 b = grid_node(g, u);
      for (int q2 = 0; q2 < 6 && !any; ++q2)
        if ((b.mask >> q2) & 1u) any |= state[u + b.off[q2]] == 1;
    }
    if (any) state[i] = 2;
    else ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(undecided, cnt);
}

__global__ void __launch_bounds__(256) agg0_phase1_k(GridGraph g,
                                                     const unsigned char* __restrict__ root,
                                                     int* __restrict__ root1) {
  SAAMG_CHUNK_LOOP {
    Nb0 r;
    if (!grid_row(g, c, lane, r)) continue;
    if (!root[r.row]) continue;
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if ((r.mask >> q) & 1u) root1[r.row + r.off[q]] = r.row;
    root1[r.row] = r.row;
  }
}

// the roots of the neighbours' phase-1 aggregates compete by priority (root ids from `ids`)
__global__ void __launch_bounds__(256) agg0_phase2_k(GridGraph g, const unsigned* __restrict__ ids,
                                                     uint32_t seed,
                                                     const int* __restrict__ root1,
                                                     int* __restrict__ aggroot,
                                                     int* __restrict__ err) {
  SAAMG_CHUNK_LOOP {
    Nb0 r;
    if (!grid_row(g, c, lane, r)) continue;
    const int own = root1[r.row];
    if (own >= 0) {
      aggroot[r.row] = own;
      continue;
    }
    unsigned long long best = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if ((r.mask >> q) & 1u) {
        const int rt = root1[r.row + r.off[q]];
        if (rt >= 0) {
          const unsigned long long k = prio(ids, rt, seed);
          best = k > best ? k : best;
        }
      }
    }
    if (best == 0) {
      aggroot[r.row] = -1;
      atomicOr(err, 1);
    } else {
      aggroot[r.row] = (int)(uint32_t)((best - 1ull) & 0xffffffffull);
    }
  }
}

#undef SAAMG_CHUNK_LOOP

// --- cubes of 3 x 3 x 3 lattice nodes ---------------------------------------------
__global__ void cube_mark_k(int n, const unsigned* __restrict__ ids, unsigned d0, unsigned d1,
                            unsigned c0, unsigned c1, int* __restrict__ cube_of,
                            unsigned char* __restrict__ used, int* __restrict__ first) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const unsigned id = ids[v];
  const unsigned i = id % d0, j = (id / d0) % d1, k = id / d0 / d1;
  const int c = (int)(i / 3 + c0 * (j / 3 + c1 * (k / 3)));
  cube_of[v] = c;
  used[c] = 1;
  atomicMin(&first[c], v);  // the minimum is the same whatever the order of the updates
}

__global__ void cube_assign_k(int n, const int* __restrict__ cube_of, const int* __restrict__ rank,
                              const int* __restrict__ first, int* __restrict__ agg,
                              unsigned char* __restrict__ root) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int c = cube_of[v];
  agg[v] = rank[c];
  root[v] = first[c] == v;
}

__global__ void cube_ids_k(int ncubes, const unsigned char* __restrict__ used,
                           const int* __restrict__ rank, unsigned* __restrict__ next_ids) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncubes && used[c]) next_ids[rank[c]] = (unsigned)c;
}

template <int G>
int rounds(int n, const int* rowptr, const int* col, const unsigned* ids, uint32_t seed,
           unsigned char* state, unsigned long long* m1, unsigned char* o1, int* counter,
           int* list, cudaStream_t s) {
  long long need = ((long long)n * G + 255) / 256;
  int blocks = (int)(need < sm_count() * 16 ? (need > 0 ? need : 1) : sm_count() * 16);
  int rounds_done = 0;
  int left = n;
  for (;;) {
    if (list && n >= 200000 && left < n / 16) {
      // few undecided rows of a large level: a round on their list (o1 holds the join flags,
      // counter[1] the list length; on small levels the full rounds are cheaper than the
      // distance-2 walks of the listed rows)
      SAAMG_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
      mis_list_k<<<(n + 255) / 256, 256, 0, s>>>(n, state, list, counter + 1);
      SAAMG_LAUNCH();
      const long long lneed = ((long long)left * G + 255) / 256;
      const int lblocks = (int)(lneed < sm_count() * 16 ? (lneed > 0 ? lneed : 1) : sm_count() * 16);
      mis_join_list_k<G><<<lblocks, 256, 0, s>>>(list, counter + 1, rowptr, col, state, ids,
                                                 seed, o1);
      SAAMG_LAUNCH();
      mis_set_list_k<<<(left + 255) / 256, 256, 0, s>>>(list, counter + 1, o1, state);
      SAAMG_LAUNCH();
      mis_leave_list_k<G><<<lblocks, 256, 0, s>>>(list, counter + 1, rowptr, col, state,
                                                  counter);
      SAAMG_LAUNCH();
      ++rounds_done;
      d2h_sync(&left, counter, sizeof(int), s);
      if (left == 0) break;
      if (rounds_done > n + 1) fail(SAAMG_NUMERICAL, "MIS-2 rounds did not terminate");
      continue;
    }
    mis_max1_k<G><<<blocks, 256, 0, s>>>(n, rowptr, col, state, ids, seed, m1);
    SAAMG_LAUNCH();
    mis_max2_k<G><<<blocks, 256, 0, s>>>(n, rowptr, col, state, ids, seed, m1);
    SAAMG_LAUNCH();
    mis_or1_k<G><<<blocks, 256, 0, s>>>(n, rowptr, col, state, o1);
    SAAMG_LAUNCH();
    SAAMG_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    mis_or2_k<G><<<blocks, 256, 0, s>>>(n, rowptr, col, state, o1, counter);
    SAAMG_LAUNCH();
    ++rounds_done;
    d2h_sync(&left, counter, sizeof(int), s);
    if (left == 0) break;
    // every round removes at least the undecided node of largest priority
    if (rounds_done > n + 1) fail(SAAMG_NUMERICAL, "MIS-2 rounds did not terminate");
  }
  return rounds_done;
}

template <int G>
void phase2(int n, const int* rowptr, const int* col, const unsigned* ids, uint32_t seed,
            const int* root1, int* aggroot, int* err, cudaStream_t s) {
  long long need = ((long long)n * G + 255) / 256;
  int blocks = (int)(need < sm_count() * 16 ? (need > 0 ? need : 1) : sm_count() * 16);
  agg_phase2_k<G><<<blocks, 256, 0, s>>>(n, rowptr, col, ids, seed, root1, aggroot, err);
  SAAMG_LAUNCH();
}

}  // namespace

int mis2_aggregate(int n, const int* rowptr, const int* col, long long nnz, const unsigned* ids,
                   uint32_t seed, unsigned char* root, int* agg, const AggScratch& w,
                   cudaStream_t s) {
  if (n <= 0) return 0;
  double avg = (double)nnz / (double)n;
  SAAMG_CUDA(cudaMemsetAsync(w.state, 0, (size_t)n, s));
  if (avg <= 8.0)
    rounds<4>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, w.list, s);
  else if (avg <= 24.0)
    rounds<8>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, w.list, s);
  else if (avg <= 64.0)
    rounds<16>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, w.list, s);
  else
    rounds<32>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, w.list, s);
  roots_from_state_k<<<(n + 255) / 256, 256, 0, s>>>(n, w.state, root);
  SAAMG_LAUNCH();
  fill_int(w.root1, -1, (size_t)n, s);
  agg_phase1_k<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, col, root, w.root1);
  SAAMG_LAUNCH();
  SAAMG_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
  if (avg <= 8.0)
    phase2<4>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  else if (avg <= 24.0)
    phase2<8>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  else if (avg <= 64.0)
    phase2<16>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  else
    phase2<32>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  long long nagg = exclusive_scan_u8(root, w.rank, n, s);
  agg_number_k<<<(n + 255) / 256, 256, 0, s>>>(n, w.aggroot, w.rank, agg);
  SAAMG_LAUNCH();
  int err = 0;
  d2h_sync(&err, w.counter, sizeof(int), s);
  if (err) fail(SAAMG_NUMERICAL, "aggregation left a node without an aggregate");
  return (int)nagg;
}

int mis2_aggregate_grid(int n, const GridGraph& g, const unsigned* ids, uint32_t seed,
                        unsigned char* root, int* agg, const AggScratch& w, cudaStream_t s) {
  if (n <= 0) return 0;
  const long long need = ((long long)g.nchunks + 7) / 8;
  const int blocks = (int)(need < sm_count() * 16 ? (need > 0 ? need : 1) : sm_count() * 16);
  SAAMG_CUDA(cudaMemsetAsync(w.state, 0, (size_t)n, s));
  for (int done = 0, left = n;;) {
    if (g.rline && w.list && n >= 200000 && left < n / 16) {
      // few undecided rows of a large level: a round on their list (o1 holds the join
      // flags, counter[1] the list length)
      SAAMG_CUDA(cudaMemsetAsync(w.counter, 0, 2 * sizeof(int), s));
      mis_list_k<<<(n + 255) / 256, 256, 0, s>>>(n, w.state, w.list, w.counter + 1);
      SAAMG_LAUNCH();
      const int lblocks = (int)std::min<long long>(((long long)left + 255) / 256, sm_count() * 16);
      mis0_join_list_k<<<lblocks, 256, 0, s>>>(w.list, w.counter + 1, g, w.state, seed, w.o1);
      SAAMG_LAUNCH();
      mis_set_list_k<<<lblocks, 256, 0, s>>>(w.list, w.counter + 1, w.o1, w.state);
      SAAMG_LAUNCH();
      mis0_leave_list_k<<<lblocks, 256, 0, s>>>(w.list, w.counter + 1, g, w.state, w.counter);
      SAAMG_LAUNCH();
      d2h_sync(&left, w.counter, sizeof(int), s);
      if (left == 0) break;
      if (++done > n + 1) fail(SAAMG_NUMERICAL, "MIS-2 rounds did not terminate");
      continue;
    }
    mis0_max1_k<<<blocks, 256, 0, s>>>(g, w.state, seed, w.m1);
    SAAMG_LAUNCH();
    mis0_max2_k<<<blocks, 256, 0, s>>>(g, w.state, seed, w.m1);
    SAAMG_LAUNCH();
    mis0_or1_k<<<blocks, 256, 0, s>>>(g, w.state, w.o1);
    SAAMG_LAUNCH();
    SAAMG_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
    mis0_or2_k<<<blocks, 256, 0, s>>>(g, w.state, w.o1, w.counter);
    SAAMG_LAUNCH();
    d2h_sync(&left, w.counter, sizeof(int), s);
    if (left == 0) break;
    if (++done > n + 1) fail(SAAMG_NUMERICAL, "MIS-2 rounds did not terminate");
  }
  roots_from_state_k<<<(n + 255) / 256, 256, 0, s>>>(n, w.state, root);
  SAAMG_LAUNCH();
  fill_int(w.root1, -1, (size_t)n, s);
  agg0_phase1_k<<<blocks, 256, 0, s>>>(g, root, w.root1);
  SAAMG_LAUNCH();
  SAAMG_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
  agg0_phase2_k<<<blocks, 256, 0, s>>>(g, ids, seed, w.root1, w.aggroot, w.counter);
  SAAMG_LAUNCH();
  long long nagg = exclusive_scan_u8(root, w.rank, n, s);
  agg_number_k<<<(n + 255) / 256, 256, 0, s>>>(n, w.aggroot, w.rank, agg);
  SAAMG_LAUNCH();
  int err = 0;
  d2h_sync(&err, w.counter, sizeof(int), s);
  if (err) fail(SAAMG_NUMERICAL, "aggregation left a node without an aggregate");
  return (int)nagg;
}

int cube_aggregate(int n, const unsigned* ids, const int dims[3], int* agg, unsigned char* root,
                   Buf<unsigned>& next_ids, int next_dims[3], cudaStream_t s) {
  const long long c0 = (dims[0] + 2) / 3, c1 = (dims[1] + 2) / 3, c2 = (dims[2] + 2) / 3;
  next_dims[0] = (int)c0;
  next_dims[1] = (int)c1;
  next_dims[2] = (int)c2;
  if (n <= 0) return 0;
  if (!ids) fail(SAAMG_EINVAL, "cube aggregation needs lattice ids");
  const long long ncubes = c0 * c1 * c2;
  if (ncubes > INT_MAX / 2) fail(SAAMG_EINVAL, "cube lattice too large");
  Buf<int> cube_of, first, rank;
  Buf<unsigned char> used;
  cube_of.alloc(n, s);
  first.alloc(ncubes, s);
  rank.alloc(ncubes, s);
  used.alloc(ncubes, s);
  SAAMG_CUDA(cudaMemsetAsync(used.p, 0, (size_t)ncubes, s));
  fill_int(first.p, INT_MAX, (size_t)ncubes, s);
  cube_mark_k<<<(n + 255) / 256, 256, 0, s>>>(n, ids, (unsigned)dims[0], (unsigned)dims[1],
                                              (unsigned)c0, (unsigned)c1, cube_of.p, used.p,
                                              first.p);
  SAAMG_LAUNCH();
  const long long nagg = exclusive_scan_u8(used.p, rank.p, (int)ncubes, s);
  cube_assign_k<<<(n + 255) / 256, 256, 0, s>>>(n, cube_of.p, rank.p, first.p, agg, root);
  SAAMG_LAUNCH();
  next_ids.alloc(nagg, s);
  cube_ids_k<<<(int)((ncubes + 255) / 256), 256, 0, s>>>((int)ncubes, used.p, rank.p,
                                                          next_ids.p);
  SAAMG_LAUNCH();
  return (int)nagg;
}

int mis2_aggregate_into(int n, const int* rowptr, const int* col, long long nnz,
                        const unsigned* ids, uint32_t seed, unsigned char* root, int* agg,
                        const AggScratch& w, long long* tiles, cudaStream_t s) {
  if (n <= 0) return 0;
  double avg = (double)nnz / (double)n;
  SAAMG_CUDA(cudaMemsetAsync(w.state, 0, (size_t)n, s));
  if (avg <= 8.0)
    rounds<4>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, nullptr, s);
  else if (avg <= 24.0)
    rounds<8>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, nullptr, s);
  else if (avg <= 64.0)
    rounds<16>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, nullptr, s);
  else
    rounds<32>(n, rowptr, col, ids, seed, w.state, w.m1, w.o1, w.counter, nullptr, s);
  roots_from_state_k<<<(n + 255) / 256, 256, 0, s>>>(n, w.state, root);
  SAAMG_LAUNCH();
  fill_int(w.root1, -1, (size_t)n, s);
  agg_phase1_k<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, col, root, w.root1);
  SAAMG_LAUNCH();
  SAAMG_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
  if (avg <= 8.0)
    phase2<4>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  else if (avg <= 24.0)
    phase2<8>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  else if (avg <= 64.0)
    phase2<16>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  else
    phase2<32>(n, rowptr, col, ids, seed, w.root1, w.aggroot, w.counter, s);
  long long nagg = exclusive_scan_u8_into(root, w.rank, n, tiles, s);
  agg_number_k<<<(n + 255) / 256, 256, 0, s>>>(n, w.aggroot, w.rank, agg);
  SAAMG_LAUNCH();
  int err = 0;
  d2h_sync(&err, w.counter, sizeof(int), s);
  if (err) fail(SAAMG_NUMERICAL, "aggregation left a node without an aggregate");
  return (int)nagg;
}

void AggScratchBufs::alloc(int n, cudaStream_t s) {
  state.alloc(n, s);
  o1.alloc(n, s);
  m1.alloc(n, s);
  counter.alloc(2, s);
  root1.alloc(n, s);
  aggroot.alloc(n, s);
  rank.alloc(n, s);
}

AggScratch AggScratchBufs::view() const {
  AggScratch w;
  w.state = state.p;
  w.o1 = o1.p;
  w.m1 = m1.p;
  w.counter = counter.p;
  w.root1 = root1.p;
  w.aggroot = aggroot.p;
  w.rank = rank.p;
  w.list = root1.p;  // the rounds' list of undecided rows (root1 is filled only afterwards)
  return w;
}

}  // namespace saamg

// ===========================================================================
// Allocation-free variant of saamg_mis2_aggregate.
//
// Some callers cannot allocate device memory at the moment they need an aggregation:
// code running inside a memory pool that must not grow, a host thread that holds a lock
// the allocator also takes, or a framework whose allocator may not be re-entered from a
// callback.  For them the scratch of the aggregation lives in one array with static
// storage on every device that loads this library (kNoallocBytes, held until the process
// exits), so the call itself allocates nothing: no cudaMalloc, cudaFree, allocator hook or
// temporary buffer.  The price is a size limit and no concurrency: calls share the array.
// ===========================================================================
namespace saamg {
namespace {

constexpr int kNoallocMaxNodes = 1 << 18;  // 262,144 graph nodes
constexpr size_t kAlignN(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffState = 0;
constexpr size_t kOffO1 = kOffState + kAlignN(kNoallocMaxNodes);
constexpr size_t kOffM1 = kOffO1 + kAlignN(kNoallocMaxNodes);
constexpr size_t kOffCounter = kOffM1 + kAlignN(sizeof(unsigned long long) * kNoallocMaxNodes);
constexpr size_t kOffRoot1 = kOffCounter + 256;
constexpr size_t kOffAggroot = kOffRoot1 + kAlignN(sizeof(int) * kNoallocMaxNodes);
constexpr size_t kOffRank = kOffAggroot + kAlignN(sizeof(int) * kNoallocMaxNodes);
constexpr size_t kOffTiles = kOffRank + kAlignN(sizeof(int) * kNoallocMaxNodes);
constexpr size_t kTileEntries = kNoallocMaxNodes / 2048 + 2;
constexpr size_t kNoallocBytes = kOffTiles + kAlignN(sizeof(long long) * kTileEntries);

// The scratch itself (about 5.8 MB).  Every call overwrites what it reads before reading
// it; nothing carries over between calls.
static __device__ __align__(256) unsigned char g_mis2_scratch[kNoallocBytes];

// Device address of the scratch in the current context.  Looked up on every call: once the
// module is loaded the lookup is a table search that allocates nothing, and a cached address
// would go stale when the device is reset and the module is loaded again at another address.
// The very first lookup on a device loads the module, which must not happen inside a stream
// capture.
unsigned char* noalloc_scratch() {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_mis2_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    fail(SAAMG_ECUDA, std::string("cudaGetSymbolAddress of the aggregation scratch: ") +
                          cudaGetErrorString(e));
  }
  return static_cast<unsigned char*>(p);
}

}  // namespace
}  // namespace saamg

extern "C" saamg_status saamg_mis2_aggregate_noalloc(int n, const int* rowptr, const int* col,
                                                     const uint32_t* ids, uint32_t seed,
                                                     unsigned char* root, int* agg, int* n_agg,
                                                     void* stream) {
  using namespace saamg;
  try {
    if (n < 0 || !n_agg) fail(SAAMG_EINVAL, "bad size or NULL n_agg");
    *n_agg = 0;
    if (n > kNoallocMaxNodes)
      fail(SAAMG_EINVAL, "graph has " + std::to_string(n) + " nodes; the allocation-free "
                         "aggregation handles at most " + std::to_string(kNoallocMaxNodes));
    if (n == 0) return SAAMG_OK;
    if (!rowptr || !col || !root || !agg) fail(SAAMG_EINVAL, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = noalloc_scratch();
    AggScratch w;
    w.state = base + kOffState;
    w.o1 = base + kOffO1;
    w.m1 = reinterpret_cast<unsigned long long*>(base + kOffM1);
    w.counter = reinterpret_cast<int*>(base + kOffCounter);
    w.root1 = reinterpret_cast<int*>(base + kOffRoot1);
    w.aggroot = reinterpret_cast<int*>(base + kOffAggroot);
    w.rank = reinterpret_cast<int*>(base + kOffRank);
    long long* tiles = reinterpret_cast<long long*>(base + kOffTiles);
    int nnz = 0;
    d2h_sync(&nnz, rowptr + n, sizeof(int), s);
    *n_agg = mis2_aggregate_into(n, rowptr, col, nnz, ids, seed, root, agg, w, tiles, s);
    SAAMG_CUDA(cudaStreamSynchronize(s));
    return SAAMG_OK;
  } catch (const Error& e) {
    set_last_error(std::string("saamg_mis2_aggregate_noalloc: ") + e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("saamg_mis2_aggregate_noalloc: out of host memory");
    return SAAMG_ENOMEM;
  } catch (...) {
    set_last_error("saamg_mis2_aggregate_noalloc: unexpected exception");
    return SAAMG_ECUDA;
  }
}
