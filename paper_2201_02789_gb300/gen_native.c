/* Native twin of gen.py's R-MAT recipe, for the large batched inputs.
 *
 * Same counter-based generator (splitmix64 finaliser over key + (i+1)*GAMMA),
 * same 16-bit quadrant fields, same redraw streams and the same CSR order
 * (sorted by (src, dst), duplicates kept), so for every argument it returns the
 * bytes gen.rmat returns; a CPU test compares the two. It draws inputs only and
 * holds none of the traversal arithmetic. Single-threaded per call; callers run
 * several instances in parallel threads. */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ull

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t stream_key(uint64_t seed, uint32_t stream) {
  return mix64(((seed & 0xFFFFFFFFull) << 32) ^ (uint64_t)stream ^ 0xD1B54A32D192ED03ull);
}

/* output i of a stream with key k */
static uint64_t draw(uint64_t k, uint64_t i) { return mix64(k + (i + 1) * GAMMA); }

/* edge `e` of an R-MAT stream: `scale` levels, field l%4 of output e*words + l/4 */
static void rmat_edge(uint64_t key, int scale, uint64_t e, uint32_t ta, uint32_t tb, uint32_t tc, uint32_t* s,
                      uint32_t* d) {
  const int words = (scale + 3) / 4;
  uint32_t src = 0, dst = 0;
  uint64_t w = 0;
  for (int l = 0; l < scale; l++) {
    if (l % 4 == 0) w = draw(key, e * (uint64_t)words + (uint64_t)(l / 4));
    const uint32_t r = (uint32_t)((w >> (16 * (l % 4))) & 0xFFFFu);
    const int shift = scale - 1 - l;
    src |= (uint32_t)(r >= tb) << shift;
    dst |= (uint32_t)((r >= ta && r < tb) || r >= tc) << shift;
  }
  *s = src;
  *d = dst;
}

/* R-MAT digraph as gen.rmat(scale, n=n, m=m, seed) with thresholds ta < tb < tc
 * (the cumulative 16-bit quadrant bounds). Writes row_ptr[n+1], col[m] and, if
 * w is not NULL, weights uniform in [wlo, whi] in CSR order. Returns 0, or -1
 * when memory runs out or the redraws do not converge. */
int npgen_rmat(int scale, int32_t n, int64_t m, uint64_t seed, uint32_t s_rmat, uint32_t s_weight, uint32_t ta,
               uint32_t tb, uint32_t tc, int32_t* row_ptr, int32_t* col, uint32_t* w, uint32_t wlo, uint32_t whi) {
  uint32_t* src = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
  uint32_t* dst = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
  int64_t* bad = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
  int rc = 0;
  if (!src || !dst || !bad || !cnt || !tmp) {
    rc = -1;
    goto out;
  }
  {
    const uint64_t key = stream_key(seed, s_rmat);
    for (int64_t e = 0; e < m; e++) rmat_edge(key, scale, (uint64_t)e, ta, tb, tc, &src[e], &dst[e]);
  }
  /* redraw self-loops and out-of-range endpoints: attempt a uses stream
   * s_rmat + 1000a under seed ^ (a * 0x51ED27), output j for the j-th bad edge
   * in increasing edge order; only redrawn edges can turn good or stay bad */
  {
    int64_t nb = 0;
    for (int64_t e = 0; e < m; e++)
      if (src[e] == dst[e] || src[e] >= (uint32_t)n || dst[e] >= (uint32_t)n) bad[nb++] = e;
    for (int attempt = 1; nb > 0; attempt++) {
      if (attempt > 10000) {
        rc = -1;
        goto out;
      }
      const uint64_t key = stream_key(seed ^ ((uint64_t)attempt * 0x51ED27ull), s_rmat + 1000u * (uint32_t)attempt);
      int64_t kept = 0;
      for (int64_t j = 0; j < nb; j++) {
        const int64_t e = bad[j];
        rmat_edge(key, scale, (uint64_t)j, ta, tb, tc, &src[e], &dst[e]);
        if (src[e] == dst[e] || src[e] >= (uint32_t)n || dst[e] >= (uint32_t)n) bad[kept++] = e;
      }
      nb = kept;
    }
  }
  /* CSR sorted by (src, dst): stable counting sort by dst, then by src */
  {
    int64_t* c = cnt;
    memset(c, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) c[dst[e] + 1]++;
    for (int64_t v = 0; v < n; v++) c[v + 1] += c[v];
    /* order by dst: tmp holds the src of each slot, bad (reused) the dst */
    for (int64_t e = 0; e < m; e++) {
      const int64_t p = c[dst[e]]++;
      tmp[p] = src[e];
      bad[p] = dst[e];
    }
    memset(c, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) c[tmp[e] + 1]++;
    for (int64_t v = 0; v < n; v++) c[v + 1] += c[v];
    for (int64_t v = 0; v <= n; v++) row_ptr[v] = (int32_t)c[v];
    for (int64_t e = 0; e < m; e++) {
      const int64_t p = c[tmp[e]]++;
      col[p] = (int32_t)bad[e];
    }
  }
  if (w) {
    const uint64_t key = stream_key(seed, s_weight);
    const uint64_t span = (uint64_t)(whi - wlo + 1);
    for (int64_t e = 0; e < m; e++) {
      const uint64_t top = draw(key, (uint64_t)e) >> 32;
      w[e] = (uint32_t)((top * span) >> 32) + wlo;
    }
  }
out:
  free(src);
  free(dst);
  free(bad);
  free(cnt);
  free(tmp);
  return rc;
}
