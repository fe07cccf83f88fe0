/*
 * ORACLE (test infrastructure only; never part of the library's compute path).
 *
 * Minimum spanning forest by Kruskal's algorithm with union-find, the plain
 * definition of the forest the Awerbuch-Shiloach method reaches (Sec. 2.3:
 * with distinct weights the minimum spanning forest is unique, Sec. 1).
 *
 * The paper assumes distinct weights (Sec. 2, Sec. 2.3).  The workloads have
 * ties, so edges are ordered strictly by (ord(w), id), id = the edge's index
 * in the input COO list.  ord() maps a float32 bit pattern to an unsigned
 * integer with the same order (-0 is taken as +0; NaN is rejected earlier);
 * for uint32 weights ord(w) = w.
 *
 * Steps, in Kruskal's order:
 *   1. key(e) = ord(w_e) * 2^32 + e for every edge that is not a self-loop;
 *   2. stable counting sort of the keys by their upper 32 bits (the ids are
 *      already ascending, so this is the full (ord, id) order);
 *   3. scan the keys in order, accepting an edge iff its endpoints lie in
 *      different union-find sets, then joining the sets;
 *   4. label(v) = the smallest vertex id in v's set.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static uint32_t ord_f32(uint32_t b) {
  if (b == 0x80000000u) b = 0u;
  return (b >> 31) ? ~b : (b ^ 0x80000000u);
}

static int32_t find_root(int32_t *up, int32_t x) {
  while (up[x] != x) {
    up[x] = up[up[x]];
    x = up[x];
  }
  return x;
}

/* Sort keys ascending by the upper 32 bits, stably, 8 bits per pass. */
static int sort_by_upper_half(uint64_t *keys, int64_t cnt) {
  uint64_t *tmp = (uint64_t *)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(uint64_t));
  if (!tmp) return -1;
  uint64_t *a = keys, *b = tmp;
  for (int shift = 32; shift < 64; shift += 8) {
    int64_t count[257];
    memset(count, 0, sizeof(count));
    for (int64_t i = 0; i < cnt; ++i) count[((a[i] >> shift) & 0xffu) + 1]++;
    for (int d = 0; d < 256; ++d) count[d + 1] += count[d];
    for (int64_t i = 0; i < cnt; ++i) b[count[(a[i] >> shift) & 0xffu]++] = a[i];
    uint64_t *t = a; a = b; b = t;
  }
  /* four passes: the result is back in `keys` */
  free(tmp);
  return 0;
}

/* Steps 3 and 4 on keys sorted in (ord, id) order; frees keys. */
static int64_t scan_and_label(int64_t n, uint64_t *keys, int64_t cnt, const int32_t *src,
                              const int32_t *dst, uint8_t *mask, int32_t *label) {
  int32_t *up = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!up) { free(keys); return -1; }
  for (int64_t v = 0; v < n; ++v) up[v] = (int32_t)v;
  int64_t chosen = 0;
  for (int64_t i = 0; i < cnt; ++i) {
    int64_t e = (int64_t)(keys[i] & 0xffffffffu);
    int32_t a = find_root(up, src[e]), b = find_root(up, dst[e]);
    if (a == b) continue;
    /* join: the smaller root id becomes the representative */
    if (a < b) up[b] = a; else up[a] = b;
    mask[e] = 1;
    ++chosen;
  }
  /* the representative is the smallest id of its set by construction, but
     compute the minimum explicitly so the label does not rely on it */
  for (int64_t v = 0; v < n; ++v) label[v] = INT32_MAX;
  for (int64_t v = 0; v < n; ++v) {
    int32_t r = find_root(up, (int32_t)v);
    if ((int32_t)v < label[r]) label[r] = (int32_t)v;
  }
  for (int64_t v = 0; v < n; ++v) label[v] = label[find_root(up, (int32_t)v)];
  free(keys);
  free(up);
  return chosen;
}

/*
 * n vertices, m edges (src[e], dst[e], weight word wbits[e]); wtype 0 = f32,
 * 1 = u32.  Writes mask[e] in {0,1} and label[v].  Returns the number of
 * forest edges, or -1 on allocation failure.
 */
int64_t oracle_kruskal(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                       const uint32_t *wbits, int wtype, uint8_t *mask, int32_t *label) {
  uint64_t *keys = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
  if (!keys) return -1;
  int64_t cnt = 0;
  for (int64_t e = 0; e < m; ++e) {
    mask[e] = 0;
    if (src[e] == dst[e]) continue;
    uint64_t o = (wtype == 0) ? ord_f32(wbits[e]) : wbits[e];
    keys[cnt++] = (o << 32) | (uint64_t)e;
  }
  if (sort_by_upper_half(keys, cnt) != 0) { free(keys); return -1; }
  return scan_and_label(n, keys, cnt, src, dst, mask, label);
}

/*
 * The same forest with steps 1 and 2 spread over `threads` threads (OpenMP
 * when compiled with it, else one thread): each thread writes the keys of a
 * contiguous range of edges at offsets from a prefix sum of the per-range
 * counts (so the keys stay in id order), and each radix pass is the usual
 * stable split: per-range digit counts, offsets ordered by (digit, range),
 * every range scattered in order.  Steps 3 and 4 are the sequential scan
 * above.  Used as a second CPU baseline; the results equal oracle_kruskal's.
 */
int64_t oracle_kruskal_mt(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                          const uint32_t *wbits, int wtype, uint8_t *mask, int32_t *label, int threads) {
  if (threads < 1) threads = 1;
  uint64_t *keys = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
  uint64_t *tmp = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
  int64_t *cnt = (int64_t *)calloc((size_t)threads * 256 + 1, sizeof(int64_t));
  if (!keys || !tmp || !cnt) { free(keys); free(tmp); free(cnt); return -1; }
  const int T = threads;
  /* step 1: the non-loop keys, in id order */
  int64_t total = 0;
#pragma omp parallel num_threads(T)
  {
#ifdef _OPENMP
    const int t = omp_get_thread_num(), nt = omp_get_num_threads();
#else
    const int t = 0, nt = 1;
#endif
    for (int tt = t; tt < T; tt += nt) {
      const int64_t lo = m * tt / T, hi = m * (tt + 1) / T;
      int64_t c = 0;
      for (int64_t e = lo; e < hi; ++e) c += src[e] != dst[e];
      cnt[tt] = c;
    }
#pragma omp barrier
#pragma omp single
    {
      int64_t run = 0;
      for (int tt = 0; tt < T; ++tt) { const int64_t c = cnt[tt]; cnt[tt] = run; run += c; }
      total = run;
    }
    for (int tt = t; tt < T; tt += nt) {
      const int64_t lo = m * tt / T, hi = m * (tt + 1) / T;
      int64_t o = cnt[tt];
      for (int64_t e = lo; e < hi; ++e) {
        mask[e] = 0;
        if (src[e] == dst[e]) continue;
        const uint64_t w = (wtype == 0) ? ord_f32(wbits[e]) : wbits[e];
        keys[o++] = (w << 32) | (uint64_t)e;
      }
    }
  }
  /* step 2: stable LSD radix passes over the upper 32 bits */
  uint64_t *a = keys, *b = tmp;
  for (int shift = 32; shift < 64; shift += 8) {
    memset(cnt, 0, (size_t)T * 256 * sizeof(int64_t));
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int tt = 0; tt < T; ++tt) {
      const int64_t lo = total * tt / T, hi = total * (tt + 1) / T;
      int64_t *c = cnt + (size_t)tt * 256;
      for (int64_t i = lo; i < hi; ++i) c[(a[i] >> shift) & 0xffu]++;
    }
    int64_t run = 0;
    for (int d = 0; d < 256; ++d)
      for (int tt = 0; tt < T; ++tt) {
        const int64_t c = cnt[(size_t)tt * 256 + d];
        cnt[(size_t)tt * 256 + d] = run;
        run += c;
      }
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int tt = 0; tt < T; ++tt) {
      const int64_t lo = total * tt / T, hi = total * (tt + 1) / T;
      int64_t *c = cnt + (size_t)tt * 256;
      for (int64_t i = lo; i < hi; ++i) b[c[(a[i] >> shift) & 0xffu]++] = a[i];
    }
    uint64_t *x = a; a = b; b = x;
  }
  /* four passes: the result is back in `keys` */
  free(tmp);
  free(cnt);
  return scan_and_label(n, keys, total, src, dst, mask, label);
}
