/*
 * Plain CPU oracle for the nested-parallel workloads of "A Compiler Framework
 * for Optimizing Dynamic Parallelism on GPUs" (arXiv 2201.02789).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this: only
 * the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code with the CUDA library.
 *
 * In the paper, thresholding, coarsening and aggregation leave the result of a
 * program unchanged (Section III-D: choosing to serialise or to launch is a
 * performance decision only; Section VI: the three passes may be applied in any
 * order and stay correct). So the oracle for every variant is the plain
 * definition of each benchmark's result, written out serially:
 *
 *   BFS  (Section VII, Table "Benchmarks and Datasets", SHOC origin):
 *        level[v] = fewest edges on a directed path src -> v, -1 if none.
 *        FIFO-queue breadth-first search.
 *   SSSP (same table, LonestarGPU origin):
 *        dist[v] = least sum of uint32 edge weights over directed paths
 *        src -> v, UINT32_MAX if none. Dijkstra with a binary heap, sums in
 *        uint64.
 *   BT   (same table, Bezier tessellation):
 *        per quadratic curve (P0, P1, P2), the curvature
 *        kappa = |P0 - 2 P1 + P2| / |P2 - P0|, the point count
 *        N = clamp(ceil(sqrt(kappa) * 64), 4, 4096), the curve-order exclusive
 *        scan of N as output offsets, and the points
 *        B(t_j) = (1-t)^2 P0 + 2 (1-t) t P1 + t^2 P2 at t_j = j / (N - 1),
 *        all in FP64 (the float inputs widen exactly). Chord of length zero:
 *        N = 4096 if the second difference is non-zero, else N = 4.
 *   TC   (the second CSR workload on the same engine; the evaluation's graph
 *        benchmarks have an adjacency-intersection child of this shape):
 *        the number of vertex triples {u, v, w} pairwise joined by edges of a
 *        simple undirected graph, each triple counted once as u < v < w.
 *
 * Build with -O2 -ffp-contract=off so that no multiply-add is contracted:
 * the point count must come out of correctly rounded IEEE operations only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ENOMEM (-1)
#define ORACLE_EOVERFLOW (-2)
#define ORACLE_EINVAL (-3)

/* ------------------------------------------------------------------ BFS */

/* Breadth-first search from src. Returns the number of reached vertices,
 * or a negative error code. */
int64_t oracle_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t src,
                   int32_t *level) {
  if (n <= 0 || src < 0 || src >= n) return ORACLE_EINVAL;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!queue) return ORACLE_ENOMEM;
  for (int32_t v = 0; v < n; v++) level[v] = -1;
  int64_t head = 0, tail = 0;
  level[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
      int32_t v = col[e];
      if (level[v] < 0) {
        level[v] = level[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return tail;
}

/* One BFS expansion from a frontier at level L, on a level array that already
 * holds levels 0..L: every out-neighbour v of a frontier vertex with
 * level[v] == -1 gets level L+1 and is listed once in next (order of first
 * discovery). Returns the number of vertices listed. */
int64_t oracle_bfs_expand(const int32_t *row_ptr, const int32_t *col, const int32_t *frontier,
                          int32_t count, int32_t L, int32_t *level, int32_t *next) {
  int64_t k = 0;
  for (int32_t i = 0; i < count; i++) {
    int32_t u = frontier[i];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
      int32_t v = col[e];
      if (level[v] == -1) {
        level[v] = L + 1;
        next[k++] = v;
      }
    }
  }
  return k;
}

/* ----------------------------------------------------------------- SSSP */

typedef struct {
  uint64_t d;
  int32_t v;
} heap_item;

static void heap_push(heap_item *h, int64_t *size, heap_item x) {
  int64_t i = (*size)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d <= x.d) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = x;
}

static heap_item heap_pop(heap_item *h, int64_t *size) {
  heap_item top = h[0];
  heap_item last = h[--(*size)];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= *size) break;
    if (c + 1 < *size && h[c + 1].d < h[c].d) c++;
    if (last.d <= h[c].d) break;
    h[i] = h[c];
    i = c;
  }
  h[i] = last;
  return top;
}

/* Dijkstra from src over uint32 weights. dist[v] = UINT32_MAX if unreachable.
 * Returns the number of reached vertices, or a negative error code. */
int64_t oracle_sssp(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w,
                    int32_t src, uint32_t *dist) {
  if (n <= 0 || src < 0 || src >= n) return ORACLE_EINVAL;
  int64_t m = row_ptr[n];
  uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
  heap_item *heap = (heap_item *)malloc(sizeof(heap_item) * (size_t)(m + 1));
  if (!d || !done || !heap) {
    free(d); free(done); free(heap);
    return ORACLE_ENOMEM;
  }
  for (int32_t v = 0; v < n; v++) d[v] = UINT64_MAX;
  int64_t size = 0, reached = 0;
  int rc = ORACLE_OK;
  d[src] = 0;
  heap_item s0 = {0, src};
  heap_push(heap, &size, s0);
  while (size > 0) {
    heap_item it = heap_pop(heap, &size);
    int32_t u = it.v;
    if (done[u]) continue;
    done[u] = 1;
    reached++;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
      int32_t v = col[e];
      uint64_t nd = d[u] + (uint64_t)w[e];
      if (nd < d[v]) {
        d[v] = nd;
        heap_item x = {nd, v};
        heap_push(heap, &size, x);
      }
    }
  }
  for (int32_t v = 0; v < n; v++) {
    if (d[v] == UINT64_MAX) {
      dist[v] = UINT32_MAX;
    } else if (d[v] >= (uint64_t)UINT32_MAX) {
      rc = ORACLE_EOVERFLOW;
      dist[v] = UINT32_MAX;
    } else {
      dist[v] = (uint32_t)d[v];
    }
  }
  free(d); free(done); free(heap);
  return rc == ORACLE_OK ? reached : rc;
}

/* One synchronous relaxation pass: out[v] = min(in[v], min over frontier
 * vertices u with an edge u->v and in[u] finite of in[u] + w(u,v)), sums in
 * uint64 and saturated at UINT32_MAX. The pass reads only `in`. */
void oracle_sssp_relax_pass(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const uint32_t *w, const int32_t *frontier, int32_t count,
                            const uint32_t *in, uint32_t *out) {
  memcpy(out, in, sizeof(uint32_t) * (size_t)n);
  for (int32_t i = 0; i < count; i++) {
    int32_t u = frontier[i];
    if (in[u] == UINT32_MAX) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
      uint64_t nd = (uint64_t)in[u] + (uint64_t)w[e];
      if (nd > (uint64_t)UINT32_MAX) nd = UINT32_MAX;
      if (nd < out[col[e]]) out[col[e]] = (uint32_t)nd;
    }
  }
}

/* --------------------------------------------------------------- Bezier */

/* Point count of one quadratic curve p = {x0,y0,x1,y1,x2,y2}. */
int32_t oracle_bezier_count(const float *p) {
  double x0 = p[0], y0 = p[1], x1 = p[2], y1 = p[3], x2 = p[4], y2 = p[5];
  double sx = (x0 - 2.0 * x1) + x2; /* second difference P0 - 2 P1 + P2 */
  double sy = (y0 - 2.0 * y1) + y2;
  double cx = x2 - x0;              /* chord P2 - P0 */
  double cy = y2 - y0;
  double s2 = sx * sx + sy * sy;
  double c2 = cx * cx + cy * cy;
  if (c2 == 0.0) return s2 > 0.0 ? 4096 : 4;
  double kappa = sqrt(s2) / sqrt(c2);
  double t = ceil(sqrt(kappa) * 64.0);
  if (t < 4.0) return 4;
  if (t > 4096.0) return 4096;
  return (int32_t)t;
}

/* Point j of a curve with N points, in FP64 (Bernstein form). */
void oracle_bezier_point(const float *p, int32_t N, int32_t j, double *xy) {
  double t = (double)j / (double)(N - 1);
  double u = 1.0 - t;
  double b0 = u * u, b1 = 2.0 * u * t, b2 = t * t;
  xy[0] = b0 * (double)p[0] + b1 * (double)p[2] + b2 * (double)p[4];
  xy[1] = b0 * (double)p[1] + b1 * (double)p[3] + b2 * (double)p[5];
}

/* Whole tessellation: counts, curve-order exclusive scan into offsets[0..ncurves]
 * and, if points != NULL, all points ([cap][2] doubles). Returns the total
 * number of points, or ORACLE_EOVERFLOW when it exceeds cap (offsets are still
 * written). */
int64_t oracle_bezier(int32_t ncurves, const float *ctrl, int32_t *offsets, double *points,
                      int64_t cap) {
  int64_t total = 0;
  for (int32_t c = 0; c < ncurves; c++) {
    offsets[c] = (int32_t)total;
    total += oracle_bezier_count(ctrl + 6 * (size_t)c);
  }
  offsets[ncurves] = (int32_t)total;
  if (!points) return total;
  if (total > cap) return ORACLE_EOVERFLOW;
  for (int32_t c = 0; c < ncurves; c++) {
    const float *p = ctrl + 6 * (size_t)c;
    int32_t N = offsets[c + 1] - offsets[c];
    for (int32_t j = 0; j < N; j++) oracle_bezier_point(p, N, j, points + 2 * ((size_t)offsets[c] + j));
  }
  return total;
}

/* ------------------------------------------------------------------- TC */

/* Triangles of a simple undirected graph given as a symmetric CSR with sorted
 * adjacency lists (no self-loops, no duplicate edges): every triple u < v < w
 * with v and w adjacent to u and w adjacent to v, counted once. Returns the
 * count, or ORACLE_EINVAL when an adjacency list is not strictly increasing. */
static int adjacent(const int32_t *row_ptr, const int32_t *col, int32_t a, int32_t b) {
  int64_t lo = row_ptr[a], hi = row_ptr[a + 1];
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] < b) lo = mid + 1;
    else hi = mid;
  }
  return lo < row_ptr[a + 1] && col[lo] == b;
}

int64_t oracle_triangles(int32_t n, const int32_t *row_ptr, const int32_t *col) {
  for (int32_t u = 0; u < n; u++)
    for (int64_t e = row_ptr[u] + 1; e < row_ptr[u + 1]; e++)
      if (col[e] <= col[e - 1]) return ORACLE_EINVAL;
  int64_t count = 0;
  for (int32_t u = 0; u < n; u++) {
    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
      const int32_t v = col[e];
      if (v <= u) continue;
      for (int64_t f = row_ptr[v]; f < row_ptr[v + 1]; f++) {
        const int32_t w = col[f];
        if (w <= v) continue;
        if (adjacent(row_ptr, col, u, w)) count++;
      }
    }
  }
  return count;
}
