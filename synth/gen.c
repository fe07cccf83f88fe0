/*
 * Seeded synthetic graph generators (COO edge lists with weights).
 *
 * This module produces inputs only: it holds none of the minimum spanning
 * forest arithmetic (no key order, no tie-breaking, no reduction).  Both the
 * CPU oracle and the CUDA library are fed from it.
 *
 * Randomness is counter based: every value is splitmix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) of a
 * (seed, stream, index) triple, so any edge can be regenerated on its own and
 * the output does not depend on the thread count.
 *
 * Weight encodings (written as raw 32-bit words):
 *   f32 in (0,1):   (2k+1) * 2^-24 with k = draw >> 41, exactly representable,
 *                   2^23 distinct values (ties occur, as in the workloads).
 *   u32 in [1,1000]: 1 + draw mod 1000.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

enum {
  ST_SRC = 1, ST_DST = 2, ST_W = 3, ST_RMAT = 4, ST_X = 5, ST_Y = 6,
  ST_BATCH_SEED = 7, ST_BATCH_N = 8, ST_BATCH_T = 9
};

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* The per-(seed, stream) part of a draw, computed once per stream by the
 * loops below; draw_at(base, i) is then synth_draw(seed, stream, i). */
static inline uint64_t draw_base(uint64_t seed, uint64_t stream) {
  return sm64_mix(seed ^ sm64_mix(stream + GOLDEN));
}

static inline uint64_t draw_at(uint64_t base, uint64_t i) {
  return sm64_mix(base + (i + 1) * GOLDEN);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t i) {
  return draw_at(draw_base(seed, stream), i);
}

static inline uint32_t below(uint64_t r, uint64_t n) {
  /* multiply-high of the top 32 bits: uniform enough in [0, n) for n <= 2^32 */
  return (uint32_t)(((r >> 32) * n) >> 32);
}

static inline uint32_t weight_word(uint64_t r, int wtype) {
  if (wtype == 0) {
    uint32_t k = (uint32_t)(r >> 41);             /* 23 bits */
    float f = (float)((2.0 * (double)k + 1.0) * (1.0 / 16777216.0));
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
  }
  return 1u + (uint32_t)(r % 1000u);
}

/* Uniform random multigraph: m draws, endpoints independent and uniform. */
void synth_er(int64_t n, int64_t m, uint64_t seed, int wtype,
              int32_t *src, int32_t *dst, uint32_t *w) {
  int64_t e;
#pragma omp parallel for schedule(static)
  for (e = 0; e < m; ++e) {
    src[e] = (int32_t)below(synth_draw(seed, ST_SRC, (uint64_t)e), (uint64_t)n);
    dst[e] = (int32_t)below(synth_draw(seed, ST_DST, (uint64_t)e), (uint64_t)n);
    w[e] = weight_word(synth_draw(seed, ST_W, (uint64_t)e), wtype);
  }
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each edge descends `scale`
 * levels of the recursive 2x2 partition, picking quadrant a (0,0), b (0,1),
 * c (1,0) or d (1,1).  Two levels are taken from each 64-bit draw.  No noise
 * and no vertex relabelling. */
void synth_rmat(int scale, int64_t m, double a, double b, double c,
                uint64_t seed, int wtype, int32_t *src, int32_t *dst,
                uint32_t *w) {
  const double two32 = 4294967296.0;
  const uint64_t ta = (uint64_t)(a * two32);
  const uint64_t tab = (uint64_t)((a + b) * two32);
  const uint64_t tabc = (uint64_t)((a + b + c) * two32);
  const int64_t per_edge = (scale + 1) / 2;
  const uint64_t base_rmat = draw_base(seed, ST_RMAT), base_w = draw_base(seed, ST_W);
  int64_t e;
#pragma omp parallel for schedule(static)
  for (e = 0; e < m; ++e) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int lev = 0; lev < scale; ++lev) {
      uint64_t x;
      if ((lev & 1) == 0) {
        r = draw_at(base_rmat, (uint64_t)(e * per_edge + lev / 2));
        x = r >> 32;
      } else {
        x = r & 0xffffffffULL;
      }
      uint32_t bu, bv;
      if (x < ta) { bu = 0; bv = 0; }
      else if (x < tab) { bu = 0; bv = 1; }
      else if (x < tabc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    src[e] = (int32_t)u;
    dst[e] = (int32_t)v;
    w[e] = weight_word(draw_at(base_w, (uint64_t)e), wtype);
  }
}

/* 3-D 7-point lattice nx*ny*nz; vertex (x,y,z) -> x + nx*(y + ny*z).
 * Edges are numbered lexicographically by (vertex, direction) with the
 * directions +x, +y, +z, skipping those that leave the box. */
int64_t synth_grid3d_count(int64_t nx, int64_t ny, int64_t nz) {
  return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
}

void synth_grid3d(int64_t nx, int64_t ny, int64_t nz, uint64_t seed, int wtype,
                  int32_t *src, int32_t *dst, uint32_t *w) {
  /* edges before plane z: every plane holds the same count */
  const int64_t per_plane = (nx - 1) * ny + nx * (ny - 1) + nx * ny;
  int64_t z;
#pragma omp parallel for schedule(static)
  for (z = 0; z < nz; ++z) {
    int64_t e = z * per_plane;
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t v = x + nx * (y + ny * z);
        if (x + 1 < nx) { src[e] = (int32_t)v; dst[e] = (int32_t)(v + 1); ++e; }
        if (y + 1 < ny) { src[e] = (int32_t)v; dst[e] = (int32_t)(v + nx); ++e; }
        if (z + 1 < nz) { src[e] = (int32_t)v; dst[e] = (int32_t)(v + nx * ny); ++e; }
      }
  }
  const int64_t m = synth_grid3d_count(nx, ny, nz);
  int64_t e;
#pragma omp parallel for schedule(static)
  for (e = 0; e < m; ++e) w[e] = weight_word(synth_draw(seed, ST_W, (uint64_t)e), wtype);
}

/* ---- 2-D random geometric graph ------------------------------------------
 * n points uniform in the unit square, edge (i,j), i<j, when the squared
 * distance is below r^2 with r = sqrt(avg_deg / (pi n)).  Edges are listed by
 * i, then by ascending j.  Weights are independent draws, not distances. */
typedef struct { double x, y; } pt2;

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* When src is NULL only counts edges.  Returns the edge count. */
static int64_t rgg_impl(int64_t n, double avg_deg, uint64_t seed, int wtype,
                        int32_t *src, int32_t *dst, uint32_t *w) {
  if (n <= 1) return 0;
  const double r = sqrt(avg_deg / (3.14159265358979323846 * (double)n));
  const double r2 = r * r;
  int64_t nc = (int64_t)floor(1.0 / r);
  if (nc < 1) nc = 1;
  if (nc > 4096) nc = 4096;
  pt2 *P = (pt2 *)malloc((size_t)n * sizeof(pt2));
  int64_t *cstart = (int64_t *)calloc((size_t)(nc * nc + 1), sizeof(int64_t));
  int32_t *cell_of = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *cand = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  for (int64_t i = 0; i < n; ++i) {
    P[i].x = (double)(synth_draw(seed, ST_X, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
    P[i].y = (double)(synth_draw(seed, ST_Y, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
    int64_t cx = (int64_t)(P[i].x * (double)nc), cy = (int64_t)(P[i].y * (double)nc);
    if (cx >= nc) cx = nc - 1;
    if (cy >= nc) cy = nc - 1;
    cell_of[i] = (int32_t)(cx + nc * cy);
    cstart[cell_of[i] + 1]++;
  }
  for (int64_t c = 0; c < nc * nc; ++c) cstart[c + 1] += cstart[c];
  int64_t *fill = (int64_t *)malloc((size_t)(nc * nc) * sizeof(int64_t));
  memcpy(fill, cstart, (size_t)(nc * nc) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) order[fill[cell_of[i]]++] = (int32_t)i;
  free(fill);
  int64_t e = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = cell_of[i] % nc, cy = cell_of[i] / nc, k = 0;
    for (int64_t dy = -1; dy <= 1; ++dy)
      for (int64_t dx = -1; dx <= 1; ++dx) {
        int64_t x = cx + dx, y = cy + dy;
        if (x < 0 || y < 0 || x >= nc || y >= nc) continue;
        int64_t c = x + nc * y;
        for (int64_t q = cstart[c]; q < cstart[c + 1]; ++q) {
          int32_t j = order[q];
          if (j <= i) continue;
          double ddx = P[i].x - P[j].x, ddy = P[i].y - P[j].y;
          if (ddx * ddx + ddy * ddy < r2) cand[k++] = j;
        }
      }
    if (src) {
      qsort(cand, (size_t)k, sizeof(int32_t), cmp_i32);
      for (int64_t q = 0; q < k; ++q) {
        src[e + q] = (int32_t)i;
        dst[e + q] = cand[q];
        w[e + q] = weight_word(synth_draw(seed, ST_W, (uint64_t)(e + q)), wtype);
      }
    }
    e += k;
  }
  free(P); free(cstart); free(cell_of); free(order); free(cand);
  return e;
}

int64_t synth_rgg_count(int64_t n, double avg_deg, uint64_t seed) {
  return rgg_impl(n, avg_deg, seed, 0, NULL, NULL, NULL);
}

void synth_rgg(int64_t n, double avg_deg, uint64_t seed, int wtype,
               int32_t *src, int32_t *dst, uint32_t *w) {
  rgg_impl(n, avg_deg, seed, wtype, src, dst, w);
}

/* ---- batch of uneven graphs ----------------------------------------------
 * Graph g: seed_g = draw(seed, BATCH_SEED, g); n_g = floor(nmin * (nmax/nmin)^U)
 * (log-uniform); type = draw(seed, BATCH_T, g) & 1: 0 = uniform random with
 * m_g = deg/2 * n_g draws, 1 = 2-D random geometric with average degree deg.
 * synth_batch_sizes fills nv[g], ne[g] and kind[g]; synth_batch_fill writes
 * the concatenated edges with LOCAL vertex ids given the offsets. */
void synth_batch_sizes(int64_t G, int64_t nmin, int64_t nmax, double deg,
                       uint64_t seed, int64_t *nv, int64_t *ne, int32_t *kind) {
  int64_t g;
  const double lr = log((double)nmax / (double)nmin);
#pragma omp parallel for schedule(dynamic, 16)
  for (g = 0; g < G; ++g) {
    double u = (double)(synth_draw(seed, ST_BATCH_N, (uint64_t)g) >> 11) * (1.0 / 9007199254740992.0);
    int64_t n = (int64_t)floor((double)nmin * exp(u * lr));
    if (n < nmin) n = nmin;
    if (n > nmax) n = nmax;
    uint64_t sg = synth_draw(seed, ST_BATCH_SEED, (uint64_t)g);
    int32_t t = (int32_t)(synth_draw(seed, ST_BATCH_T, (uint64_t)g) & 1u);
    nv[g] = n;
    kind[g] = t;
    ne[g] = (t == 0) ? (int64_t)(deg * 0.5 * (double)n) : synth_rgg_count(n, deg, sg);
  }
}

void synth_batch_fill(int64_t G, double deg, uint64_t seed, int wtype,
                      const int64_t *nv, const int64_t *eoff, const int32_t *kind,
                      int32_t *src, int32_t *dst, uint32_t *w) {
  int64_t g;
#pragma omp parallel for schedule(dynamic, 8)
  for (g = 0; g < G; ++g) {
    uint64_t sg = synth_draw(seed, ST_BATCH_SEED, (uint64_t)g);
    int64_t o = eoff[g], m = eoff[g + 1] - eoff[g];
    if (kind[g] == 0)
      synth_er(nv[g], m, sg, wtype, src + o, dst + o, w + o);
    else
      synth_rgg(nv[g], deg, sg, wtype, src + o, dst + o, w + o);
  }
}
