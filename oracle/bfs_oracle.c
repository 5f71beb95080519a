/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, serial, obviously correct statement of what the BFS library computes.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use it;
 * the library itself never calls, links or loads anything from this directory.
 * It shares no code with the CUDA path.
 *
 * What it computes (the plain definitions the paper's method reaches exactly):
 *   - graph: the undirected graph of an edge list, stored as CSR with each
 *     undirected edge stored in both rows, rows sorted ascending, self-loops
 *     and repeated pairs dropped (Sec. 4.1 "Graph Representation"; the
 *     benchmark symmetrises its input, Sec. 6).
 *   - level[v] = d(s, v), the hop distance from s (Sec. 2.1, Algorithm 1), or -1
 *     when v is unreachable (the int32 stand-in for Algorithm 1's infinity).
 *   - parent[s] = s; for reached v != s, parent[v] = the largest id u adjacent to
 *     v with level[u] = level[v] - 1.  This is the (select2nd, max) semiring
 *     product of Sec. 3.2 / Algorithm 3 with frontier values equal to the
 *     vertices' own ids; parent[v] = -1 when v is unreachable (Algorithm 3's
 *     output contract).
 *   - TEPS edge count of a traversal: the undirected edges inside the reached
 *     component, half the degree sum of the reached vertices (Sec. 6).
 *   - directed graphs (the paper's matrix A of Sec. 3.2 need not be symmetric;
 *     the traversal then multiplies by A^T): rows hold out-neighbours only,
 *     level[v] is the length of the shortest directed path s -> v, and
 *     parent[v] the largest id u with an arc u -> v and level[u] = level[v] - 1.
 *
 * Algorithm: the queue-based serial BFS the paper contrasts with its two-stack
 * Algorithm 1 (Sec. 2.1 -- both give the same levels), followed by a separate
 * pass that applies the max-id parent definition vertex by vertex.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int oracle_cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Builds the symmetric CSR of an edge list.
 *   offsets: int64[n+1] (written), adj: int32 scratch of capacity 2*m; on return
 *   its first nnz entries hold the rows.  Returns nnz, or -1 on a bad argument
 *   (an endpoint outside [0, n)).
 * Steps: count both directions of every non-loop edge per row, prefix-sum the
 * counts into row starts, scatter, sort every row, drop repeats within each row
 * and pack the rows to the front.
 */
int64_t oracle_build_csr(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                         int64_t* offsets, int32_t* adj) {
  if (n < 0 || m < 0 || !offsets || (m > 0 && (!src || !dst || !adj))) return -1;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;

  int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!fill) return -1;
  for (int64_t i = 0; i <= n; ++i) offsets[i] = 0;
  for (int64_t e = 0; e < m; ++e) {
    if (src[e] == dst[e]) continue;
    offsets[src[e] + 1] += 1;
    offsets[dst[e] + 1] += 1;
  }
  for (int64_t v = 0; v < n; ++v) offsets[v + 1] += offsets[v];
  for (int64_t v = 0; v < n; ++v) fill[v] = offsets[v];
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u == v) continue;
    adj[fill[u]++] = v;
    adj[fill[v]++] = u;
  }
  /* sort each row and drop repeats; rows are packed towards the front */
  int64_t out = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t b = offsets[v], e = offsets[v + 1];
    qsort(adj + b, (size_t)(e - b), sizeof(int32_t), oracle_cmp_i32);
    int64_t row_start = out;
    for (int64_t i = b; i < e; ++i) {
      if (i > b && adj[i] == adj[i - 1]) continue;
      adj[out++] = adj[i];
    }
    offsets[v] = row_start;
  }
  offsets[n] = out;
  free(fill);
  return out;
}

/*
 * Serial BFS from s.  level, parent: int32[n] (written); queue: int32[n] scratch.
 * Returns the number of levels (1 + the largest finite level), or -1 on a bad
 * argument.
 */
int32_t oracle_bfs(const int64_t* offsets, const int32_t* adj, int32_t n, int32_t s,
                   int32_t* level, int32_t* parent, int32_t* queue) {
  if (n <= 0 || s < 0 || s >= n || !offsets || !level || !parent || !queue) return -1;
  for (int32_t v = 0; v < n; ++v) {
    level[v] = -1;
    parent[v] = -1;
  }
  /* levels: FIFO queue, each vertex gets level[u] + 1 the first time it is seen */
  int64_t head = 0, tail = 0;
  level[s] = 0;
  queue[tail++] = s;
  int32_t deepest = 0;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t i = offsets[u]; i < offsets[u + 1]; ++i) {
      int32_t v = adj[i];
      if (level[v] == -1) {
        level[v] = level[u] + 1;
        if (level[v] > deepest) deepest = level[v];
        queue[tail++] = v;
      }
    }
  }
  /* parents: the largest neighbour one level closer to s */
  parent[s] = s;
  for (int32_t v = 0; v < n; ++v) {
    if (level[v] <= 0) continue;
    int32_t best = -1;
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i) {
      int32_t u = adj[i];
      if (level[u] == level[v] - 1 && u > best) best = u;
    }
    parent[v] = best;
  }
  return deepest + 1;
}

/* Undirected edges inside the reached set: half the degree sum of reached vertices. */
int64_t oracle_component_edges(const int64_t* offsets, const int32_t* level, int32_t n) {
  int64_t sum = 0;
  for (int32_t v = 0; v < n; ++v)
    if (level[v] >= 0) sum += offsets[v + 1] - offsets[v];
  return sum / 2;
}

/*
 * Per-level frontier statistics of a finished traversal: for k < nlevels,
 * count[k] = |{v : level[v] = k}| and edges[k] = sum of their degrees.
 */
int oracle_level_stats(const int64_t* offsets, const int32_t* level, int32_t n, int32_t nlevels,
                       int64_t* count, int64_t* edges) {
  if (nlevels < 0 || !count || !edges) return -1;
  for (int32_t k = 0; k < nlevels; ++k) count[k] = edges[k] = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t k = level[v];
    if (k < 0 || k >= nlevels) continue;
    count[k] += 1;
    edges[k] += offsets[v + 1] - offsets[v];
  }
  return 0;
}

/*
 * Checks a BFS result against an edge list, in O(m + n), without building a
 * CSR.  The result is accepted when
 *   (a) level[s] = 0 and parent[s] = s;
 *   (b) for every non-loop edge (u, v): level[u] = -1 exactly when level[v] = -1,
 *       and |level[u] - level[v]| <= 1;
 *   (c) every reached v != s has a neighbour one level closer to s, and
 *       parent[v] is the largest such neighbour; unreached vertices have
 *       parent -1.
 * (a)-(c) make level the hop distance: following parents gives a path of
 * length level[v], so d(s, v) <= level[v]; along any path from s the level
 * grows by at most one per edge, so level[v] <= d(s, v).  (c) is the max-id
 * parent rule of Sec. 3.2 itself.
 * best: int32 scratch[n].  bad[0..3] receive the violations of (a), (b),
 * (c)-parent and (c)-unreached; returns their sum, or -1 on a bad argument.
 */
int64_t oracle_validate_edges(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, int32_t s,
                              const int32_t* level, const int32_t* parent, int32_t* best, int64_t* bad) {
  if (n <= 0 || s < 0 || s >= n || !level || !parent || !best || !bad || (m > 0 && (!src || !dst))) return -1;
  for (int i = 0; i < 4; ++i) bad[i] = 0;
  if (level[s] != 0 || parent[s] != s) bad[0] += 1;
  for (int32_t v = 0; v < n; ++v) best[v] = -1;
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) return -1;
    if (u == v) continue;
    int32_t lu = level[u], lv = level[v];
    if ((lu < 0) != (lv < 0)) {
      bad[1] += 1;
      continue;
    }
    if (lu < 0) continue;
    if (lu - lv > 1 || lv - lu > 1) bad[1] += 1;
    if (lu == lv - 1 && u > best[v]) best[v] = u;
    if (lv == lu - 1 && v > best[u]) best[u] = v;
  }
  for (int32_t v = 0; v < n; ++v) {
    if (v == s) continue;
    if (level[v] > 0) {
      if (best[v] < 0 || parent[v] != best[v]) bad[2] += 1;
    } else if (level[v] == 0 || parent[v] != -1 || level[v] < -1) {
      bad[3] += 1;
    }
  }
  return bad[0] + bad[1] + bad[2] + bad[3];
}

/*
 * Directed CSR of an edge list: row u holds the heads v of the arcs u -> v,
 * sorted, repeats and self-loops dropped.  offsets: int64[n+1], adj: int32
 * scratch of capacity m.  Returns nnz, or -1 on a bad argument.
 */
int64_t oracle_build_digraph_csr(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                                 int64_t* offsets, int32_t* adj) {
  if (n < 0 || m < 0 || !offsets || (m > 0 && (!src || !dst || !adj))) return -1;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
  int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!fill) return -1;
  for (int64_t i = 0; i <= n; ++i) offsets[i] = 0;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) offsets[src[e] + 1] += 1;
  for (int64_t v = 0; v < n; ++v) offsets[v + 1] += offsets[v];
  for (int64_t v = 0; v < n; ++v) fill[v] = offsets[v];
  for (int64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) adj[fill[src[e]]++] = dst[e];
  int64_t out = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t b = offsets[v], e = offsets[v + 1];
    qsort(adj + b, (size_t)(e - b), sizeof(int32_t), oracle_cmp_i32);
    int64_t row_start = out;
    for (int64_t i = b; i < e; ++i) {
      if (i > b && adj[i] == adj[i - 1]) continue;
      adj[out++] = adj[i];
    }
    offsets[v] = row_start;
  }
  offsets[n] = out;
  free(fill);
  return out;
}

/*
 * Serial BFS from s over the out-rows of a directed CSR; the parent pass runs
 * over every arc u -> v and keeps, for each v, the largest u one level closer.
 * Same outputs and return value as oracle_bfs.
 */
int32_t oracle_bfs_directed(const int64_t* offsets, const int32_t* adj, int32_t n, int32_t s,
                            int32_t* level, int32_t* parent, int32_t* queue) {
  if (n <= 0 || s < 0 || s >= n || !offsets || !level || !parent || !queue) return -1;
  for (int32_t v = 0; v < n; ++v) {
    level[v] = -1;
    parent[v] = -1;
  }
  int64_t head = 0, tail = 0;
  level[s] = 0;
  queue[tail++] = s;
  int32_t deepest = 0;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t i = offsets[u]; i < offsets[u + 1]; ++i) {
      int32_t v = adj[i];
      if (level[v] == -1) {
        level[v] = level[u] + 1;
        if (level[v] > deepest) deepest = level[v];
        queue[tail++] = v;
      }
    }
  }
  for (int32_t u = 0; u < n; ++u) {
    if (level[u] < 0) continue;
    for (int64_t i = offsets[u]; i < offsets[u + 1]; ++i) {
      int32_t v = adj[i];
      if (v != s && level[v] == level[u] + 1 && u > parent[v]) parent[v] = u;
    }
  }
  parent[s] = s;
  return deepest + 1;
}

/* Arcs leaving the reached set (the TEPS count of a directed traversal). */
int64_t oracle_out_edges(const int64_t* offsets, const int32_t* level, int32_t n) {
  int64_t sum = 0;
  for (int32_t v = 0; v < n; ++v)
    if (level[v] >= 0) sum += offsets[v + 1] - offsets[v];
  return sum;
}

/*
 * O(m + n) check of a directed BFS result against an arc list (u -> v), the
 * directed counterpart of oracle_validate_edges.  best: int32[n] scratch;
 * bad[4] receives (a) a wrong source entry, (b) arcs u -> v with u reached and
 * v unreached or level[v] > level[u] + 1, (c) reached v != s without an
 * in-neighbour one level up, or with a parent other than the largest such
 * in-neighbour, or at level 0, (d) unreached v with parent != -1 or a level
 * below -1.  All four are zero exactly when level[] are the directed distances
 * from s and parent[] follows the max-id rule: (b) bounds every level by the
 * distance and closes the reached set under the arcs, (c) gives every reached
 * vertex a path from s of its level's length.  Returns the total, -1 on a bad
 * argument.
 */
int64_t oracle_validate_arcs(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, int32_t s,
                             const int32_t* level, const int32_t* parent, int32_t* best, int64_t* bad) {
  if (n <= 0 || s < 0 || s >= n || !level || !parent || !best || !bad || (m > 0 && (!src || !dst))) return -1;
  for (int i = 0; i < 4; ++i) bad[i] = 0;
  if (level[s] != 0 || parent[s] != s) bad[0] += 1;
  for (int32_t v = 0; v < n; ++v) best[v] = -1;
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) return -1;
    if (u == v || level[u] < 0) continue;
    if (level[v] < 0 || level[v] > level[u] + 1) {
      bad[1] += 1;
      continue;
    }
    if (level[v] == level[u] + 1 && u > best[v]) best[v] = u;
  }
  for (int32_t v = 0; v < n; ++v) {
    if (v == s) continue;
    if (level[v] >= 0) {
      if (level[v] == 0 || best[v] < 0 || parent[v] != best[v]) bad[2] += 1;
    } else if (parent[v] != -1 || level[v] < -1) {
      bad[3] += 1;
    }
  }
  return bad[0] + bad[1] + bad[2] + bad[3];
}
