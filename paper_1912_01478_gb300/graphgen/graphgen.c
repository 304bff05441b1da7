/*
 * Seeded synthetic graph generators and CSR tools (host C, no CUDA).
 *
 * This module only makes inputs. It holds none of the colouring method's
 * arithmetic, and both the CPU oracle's tests and the GPU path consume the
 * byte-identical graphs it produces. Every graph it returns is undirected,
 * symmetric, free of self-loops and duplicate edges, and has each CSR row
 * sorted ascending (the paper removes self loops and multi-edges from its
 * inputs before colouring them, Section V).
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018), its 256-bit state
 * filled from the seed by splitmix64 (Steele, Lea & Flood, 2014), both written
 * here from their published definitions. Integers in [0, k) take the high
 * 64 bits of a 64x64-bit product (Lemire's multiply-shift, without the
 * rejection step, so a bias of at most k/2^64); doubles in [0,1) take the top
 * 53 bits. All arithmetic is integer or IEEE double, so the output is the same
 * on x86-64 and aarch64.
 *
 * Memory returned through ipgc_gen_csr / ipgc_gen_batch_t is malloc()ed
 * here and released with ipgc_gen_free_csr / ipgc_gen_free_batch. The C ABI
 * is declared in include/ipgc_graphgen.h.
 */
#include "ipgc_graphgen.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG -- */

typedef struct {
  uint64_t s[4];
} rng_t;

static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static void rng_seed(rng_t* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_u64(rng_t* r) {
  uint64_t* s = r->s;
  const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

static inline uint64_t rng_below(rng_t* r, uint64_t k) {
  return (uint64_t)(((unsigned __int128)rng_u64(r) * (unsigned __int128)k) >> 64);
}

static inline double rng_unit(rng_t* r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }

uint64_t ipgc_gen_derive_seed(uint64_t seed, uint64_t index) {
  uint64_t x = seed ^ (0xd1b54a32d192ed03ULL * (index + 1));
  splitmix64(&x);
  return splitmix64(&x);
}

/* ------------------------------------------------------ edge list -> CSR -- */

/* sort a short int32 run ascending (insertion sort; qsort above 32) */
static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

static void sort_run(int32_t* p, int64_t len) {
  if (len > 32) {
    qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
    return;
  }
  for (int64_t i = 1; i < len; ++i) {
    int32_t x = p[i];
    int64_t j = i - 1;
    while (j >= 0 && p[j] > x) {
      p[j + 1] = p[j];
      --j;
    }
    p[j + 1] = x;
  }
}

/*
 * Build a symmetric, self-loop-free, duplicate-free CSR with sorted rows from
 * m undirected pairs (src[e], dst[e]): count degrees, scatter both directed
 * entries of every pair into their rows (in any order), sort every row, drop
 * adjacent duplicates and compact. The result does not depend on the order
 * of the scatter, so the passes may run on several host threads.
 */
static int build_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, ipgc_gen_csr* out) {
  memset(out, 0, sizeof(*out));
  out->n = n;
  int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* pos = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t* rowptr = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  if (!start || !pos || !rowptr) {
    free(start);
    free(pos);
    free(rowptr);
    return IPGC_GEN_ERR_OOM;
  }
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u == v) continue;
#pragma omp atomic
    start[u + 1]++;
#pragma omp atomic
    start[v + 1]++;
  }
  for (int32_t v = 0; v < n; ++v) start[v + 1] += start[v];
  int64_t tot = start[n];
  int32_t* col = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
  if (!col) {
    free(start);
    free(pos);
    free(rowptr);
    return IPGC_GEN_ERR_OOM;
  }
  memcpy(pos, start, ((size_t)n + 1) * sizeof(int64_t));
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u == v) continue;
    int64_t a, b;
#pragma omp atomic capture
    a = pos[u]++;
#pragma omp atomic capture
    b = pos[v]++;
    col[a] = v;
    col[b] = u;
  }
  /* sort + dedup every row in place; pos[v] becomes the unique count */
#pragma omp parallel for schedule(dynamic, 4096)
  for (int32_t v = 0; v < n; ++v) {
    int64_t b = start[v], len = start[v + 1] - b;
    int32_t* row = col + b;
    sort_run(row, len);
    int64_t w = 0;
    for (int64_t k = 0; k < len; ++k)
      if (w == 0 || row[k] != row[w - 1]) row[w++] = row[k];
    pos[v] = w;
  }
  int64_t acc = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (acc > INT32_MAX) break;
    rowptr[v] = (int32_t)acc;
    acc += pos[v];
  }
  if (acc > INT32_MAX) {
    free(start);
    free(pos);
    free(rowptr);
    free(col);
    return IPGC_GEN_ERR_TOO_BIG;
  }
  rowptr[n] = (int32_t)acc;
  /* compact rows towards the front (destination never overtakes source) */
  for (int32_t v = 0; v < n; ++v)
    if (rowptr[v] != start[v] && pos[v] > 0)
      memmove(col + rowptr[v], col + start[v], (size_t)pos[v] * sizeof(int32_t));
  free(start);
  free(pos);
  int32_t* shrunk = (int32_t*)realloc(col, (size_t)(acc > 0 ? acc : 1) * sizeof(int32_t));
  out->rowptr = rowptr;
  out->col = shrunk ? shrunk : col;
  out->nnz = acc;
  return IPGC_GEN_OK;
}

int ipgc_gen_from_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, ipgc_gen_csr* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (n < 0 || m < 0 || !out) return IPGC_GEN_ERR_ARG;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return IPGC_GEN_ERR_ARG;
  return build_csr(n, m, src, dst, out);
}

/* ---------------------------------------------------------- generators -- */

/*
 * Erdos-Renyi G(n, m): exactly m distinct undirected edges, each drawn as a
 * uniform pair u != v, redrawn when it is a self-loop or already present
 * (open-addressing hash set over the canonical pair).
 */
static int er_edges(rng_t* r, int32_t n, int64_t m, int32_t* src, int32_t* dst) {
  uint64_t cap = 16;
  while (cap < (uint64_t)m * 2 + 16) cap <<= 1;
  uint64_t* tab = (uint64_t*)malloc(cap * sizeof(uint64_t));
  if (!tab) return IPGC_GEN_ERR_OOM;
  memset(tab, 0xff, cap * sizeof(uint64_t));
  const uint64_t EMPTY = ~0ULL;
  for (int64_t e = 0; e < m;) {
    int32_t u = (int32_t)rng_below(r, (uint64_t)n);
    int32_t v = (int32_t)rng_below(r, (uint64_t)n);
    if (u == v) continue;
    uint64_t a = (uint64_t)(u < v ? u : v), b = (uint64_t)(u < v ? v : u);
    uint64_t key = (a << 32) | b;
    uint64_t h = (key * 0x9e3779b97f4a7c15ULL) & (cap - 1);
    int dup = 0;
    while (tab[h] != EMPTY) {
      if (tab[h] == key) {
        dup = 1;
        break;
      }
      h = (h + 1) & (cap - 1);
    }
    if (dup) continue;
    tab[h] = key;
    src[e] = u;
    dst[e] = v;
    ++e;
  }
  free(tab);
  return IPGC_GEN_OK;
}

int ipgc_gen_er(uint64_t seed, int32_t n, int64_t m, ipgc_gen_csr* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (!out || n < 0 || m < 0) return IPGC_GEN_ERR_ARG;
  if (n < 2 && m > 0) return IPGC_GEN_ERR_ARG;
  if ((double)m > 0.5 * (double)n * (double)(n - 1)) return IPGC_GEN_ERR_ARG;
  rng_t r;
  rng_seed(&r, seed);
  int32_t* src = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!src || !dst) {
    free(src);
    free(dst);
    return IPGC_GEN_ERR_OOM;
  }
  int rc = er_edges(&r, n, m, src, dst);
  if (rc == IPGC_GEN_OK) rc = build_csr(n, m, src, dst, out);
  free(src);
  free(dst);
  return rc;
}

/*
 * One RMAT endpoint pair: at every level a 53-bit uniform x picks quadrant
 * a (x < A), b (A <= x < AB: column bit), c (AB <= x < ABC: row bit) or
 * d (x >= ABC: both bits), the thresholds being the probabilities scaled
 * to 2^53.
 */
static inline void rmat_pair(rng_t* r, int scale, uint64_t A, uint64_t AB, uint64_t ABC,
                             int32_t* pu, int32_t* pv) {
  uint32_t u = 0, v = 0;
  for (int lvl = scale - 1; lvl >= 0; --lvl) {
    uint64_t x = rng_u64(r) >> 11;
    uint32_t ub = (uint32_t)(x >= AB);
    uint32_t vb = (uint32_t)((x >= A) & (x < AB)) | (uint32_t)(x >= ABC);
    u |= ub << lvl;
    v |= vb << lvl;
  }
  *pu = (int32_t)u;
  *pv = (int32_t)v;
}

/* Fisher-Yates permutation of [0, n) */
static int32_t* fisher_yates(rng_t* r, int32_t n) {
  int32_t* p = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!p) return NULL;
  for (int32_t i = 0; i < n; ++i) p[i] = i;
  for (int32_t i = n - 1; i > 0; --i) {
    int32_t j = (int32_t)rng_below(r, (uint64_t)i + 1);
    int32_t t = p[i];
    p[i] = p[j];
    p[j] = t;
  }
  return p;
}

/*
 * RMAT (Chakrabarti, Zhan & Faloutsos, 2004) without noise: nedges directed
 * draws over a 2^scale square, then symmetrised and deduplicated. The draws
 * come from per-chunk streams (2^16 edges per chunk), so they are the same
 * for any number of host threads. With
 * n_limit in (0, 2^scale) the node count is n_limit and any draw with an
 * endpoint >= n_limit is redrawn whole. With permute != 0 the node IDs are
 * relabelled by a Fisher-Yates permutation drawn after the edges.
 */
int ipgc_gen_rmat(uint64_t seed, int32_t scale, int64_t nedges, double a, double b, double c,
            int32_t n_limit, int32_t permute, ipgc_gen_csr* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (!out || scale < 0 || scale > 30 || nedges < 0) return IPGC_GEN_ERR_ARG;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return IPGC_GEN_ERR_ARG;
  int32_t full = (int32_t)1 << scale;
  int32_t n = (n_limit > 0 && n_limit < full) ? n_limit : full;
  rng_t r; /* main stream: only the permutation */
  rng_seed(&r, seed);
  int32_t* src = (int32_t*)malloc((size_t)(nedges > 0 ? nedges : 1) * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)(nedges > 0 ? nedges : 1) * sizeof(int32_t));
  if (!src || !dst) {
    free(src);
    free(dst);
    return IPGC_GEN_ERR_OOM;
  }
  const double two53 = 9007199254740992.0;
  const uint64_t A = (uint64_t)(a * two53), AB = (uint64_t)((a + b) * two53),
                 ABC = (uint64_t)((a + b + c) * two53);
  /* draws come in chunks of 2^16 edges, chunk k from stream derive(seed, k) */
  const int64_t CH = (int64_t)1 << 16;
  int64_t nch = (nedges + CH - 1) / CH;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nch; ++k) {
    rng_t cr;
    rng_seed(&cr, ipgc_gen_derive_seed(seed, (uint64_t)k));
    int64_t e1 = (k + 1) * CH < nedges ? (k + 1) * CH : nedges;
    for (int64_t e = k * CH; e < e1; ++e) {
      int32_t u, v;
      do {
        rmat_pair(&cr, scale, A, AB, ABC, &u, &v);
      } while (u >= n || v >= n);
      src[e] = u;
      dst[e] = v;
    }
  }
  if (permute) {
    int32_t* p = fisher_yates(&r, n);
    if (!p) {
      free(src);
      free(dst);
      return IPGC_GEN_ERR_OOM;
    }
    for (int64_t e = 0; e < nedges; ++e) {
      src[e] = p[src[e]];
      dst[e] = p[dst[e]];
    }
    free(p);
  }
  int rc = build_csr(n, nedges, src, dst, out);
  free(src);
  free(dst);
  return rc;
}

/*
 * Road-network-like graph: a side x side 4-neighbour grid with row-major IDs
 * (node = row * side + column, not permuted). Every grid edge is deleted
 * independently with probability p_delete (visiting horizontal edges row by
 * row, then vertical edges row by row); then round(frac_long * retained)
 * long-range edges with uniform endpoints (self-loops redrawn) are added.
 * Duplicates among the long-range edges are removed by the CSR build.
 */
int ipgc_gen_road(uint64_t seed, int32_t side, double p_delete, double frac_long, ipgc_gen_csr* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (!out || side < 0 || side > 46340 || p_delete < 0 || p_delete > 1 || frac_long < 0)
    return IPGC_GEN_ERR_ARG;
  int32_t n = side * side;
  int64_t grid = side > 0 ? 2LL * side * (side - 1) : 0;
  int64_t cap = grid + (int64_t)(frac_long * (double)grid) + 16;
  int32_t* src = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  if (!src || !dst) {
    free(src);
    free(dst);
    return IPGC_GEN_ERR_OOM;
  }
  rng_t r;
  rng_seed(&r, seed);
  int64_t m = 0;
  for (int32_t row = 0; row < side; ++row)
    for (int32_t c = 0; c + 1 < side; ++c)
      if (!(rng_unit(&r) < p_delete)) {
        src[m] = row * side + c;
        dst[m] = row * side + c + 1;
        ++m;
      }
  for (int32_t row = 0; row + 1 < side; ++row)
    for (int32_t c = 0; c < side; ++c)
      if (!(rng_unit(&r) < p_delete)) {
        src[m] = row * side + c;
        dst[m] = (row + 1) * side + c;
        ++m;
      }
  int64_t nlong = (int64_t)llround(frac_long * (double)m);
  if (n < 2) nlong = 0;
  for (int64_t k = 0; k < nlong; ++k) {
    int32_t u, v;
    do {
      u = (int32_t)rng_below(&r, (uint64_t)n);
      v = (int32_t)rng_below(&r, (uint64_t)n);
    } while (u == v);
    src[m] = u;
    dst[m] = v;
    ++m;
  }
  int rc = build_csr(n, m, src, dst, out);
  free(src);
  free(dst);
  return rc;
}

/*
 * Random geometric graph: n points uniform in the unit square (dim 2) or cube
 * (dim 3), an edge between every two points at Euclidean distance < r, r set
 * so the mean degree away from the border is avg_degree (pi r^2 n in 2-D,
 * 4/3 pi r^3 n in 3-D). Points are numbered in the order of the grid cells of
 * side >= r they fall in (x fastest, then y, then z), so nearby points have
 * nearby IDs, as in the rgg graphs of the DIMACS collection. Coordinates come
 * from per-chunk streams (2^16 points per chunk).
 */
int ipgc_gen_rgg(uint64_t seed, int32_t n, int32_t dim, double avg_degree, ipgc_gen_csr* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (!out || n < 0 || (dim != 2 && dim != 3) || !(avg_degree >= 0)) return IPGC_GEN_ERR_ARG;
  const double pi = 3.14159265358979323846;
  const double r = dim == 2 ? sqrt(avg_degree / (pi * (n > 0 ? n : 1)))
                            : cbrt(3.0 * avg_degree / (4.0 * pi * (n > 0 ? n : 1)));
  int64_t G = r > 0 ? (int64_t)floor(1.0 / r) : 1;
  if (G < 1) G = 1;
  if (dim == 2 && G > 46340) G = 46340;
  if (dim == 3 && G > 1290) G = 1290;
  const int64_t ncell = dim == 2 ? G * G : G * G * G;
  double* pt = (double*)malloc(sizeof(double) * (size_t)dim * (size_t)(n > 0 ? n : 1));
  double* sp = (double*)malloc(sizeof(double) * (size_t)dim * (size_t)(n > 0 ? n : 1));
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cstart = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!pt || !sp || !cell || !cstart || !cnt) {
    free(pt); free(sp); free(cell); free(cstart); free(cnt);
    return IPGC_GEN_ERR_OOM;
  }
  const int64_t chunk = 1 << 16, nch = ((int64_t)n + chunk - 1) / chunk;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nch; ++k) {
    rng_t rr;
    rng_seed(&rr, ipgc_gen_derive_seed(seed, (uint64_t)k));
    const int64_t hi = (k + 1) * chunk < n ? (k + 1) * chunk : n;
    for (int64_t i = k * chunk; i < hi; ++i) {
      int64_t c = 0, mul = 1;
      for (int d = 0; d < dim; ++d) {
        const double x = rng_unit(&rr);
        pt[i * dim + d] = x;
        int64_t q = (int64_t)(x * (double)G);
        if (q >= G) q = G - 1;
        c += q * mul;
        mul *= G;
      }
      cell[i] = c;
    }
  }
  /* counting sort by cell: the new ID of point i is its place in cell order */
  for (int64_t i = 0; i < n; ++i) cstart[cell[i] + 1]++;
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    if (!fill) {
      free(pt); free(sp); free(cell); free(cstart); free(cnt);
      return IPGC_GEN_ERR_OOM;
    }
    memcpy(fill, cstart, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t k = fill[cell[i]]++;
      for (int d = 0; d < dim; ++d) sp[k * dim + d] = pt[i * dim + d];
    }
    free(fill);
  }
  free(pt);
  /* pairs (i, j), j > i, at distance < r: count per point, then emit */
  const double r2 = r * r;
  for (int pass = 0; pass < 2; ++pass) {
    int32_t* src = NULL;
    int32_t* dst = NULL;
    if (pass == 1) {
      cnt[0] = 0;
      for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
      src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
      dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
      if (!src || !dst) {
        free(src); free(dst); free(sp); free(cell); free(cstart); free(cnt);
        return IPGC_GEN_ERR_OOM;
      }
    }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
      int64_t q[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        q[d] = (int64_t)(sp[i * dim + d] * (double)G);
        if (q[d] >= G) q[d] = G - 1;
      }
      int64_t k = 0, w = pass ? cnt[i] : 0;
      const int64_t zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
      for (int64_t dz = zlo; dz <= zhi; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
          for (int64_t dx = -1; dx <= 1; ++dx) {
            const int64_t cx = q[0] + dx, cy = q[1] + dy, cz = q[2] + dz;
            if (cx < 0 || cy < 0 || cz < 0 || cx >= G || cy >= G || (dim == 3 && cz >= G)) continue;
            const int64_t c = cx + G * (cy + G * cz);
            for (int64_t j = cstart[c] > i + 1 ? cstart[c] : i + 1; j < cstart[c + 1]; ++j) {
              double s2 = 0;
              for (int d = 0; d < dim; ++d) {
                const double t = sp[j * dim + d] - sp[i * dim + d];
                s2 += t * t;
              }
              if (s2 < r2) {
                if (pass) {
                  src[w] = (int32_t)i;
                  dst[w] = (int32_t)j;
                  ++w;
                }
                ++k;
              }
            }
          }
      if (!pass) cnt[i + 1] = k;
    }
    if (pass == 1) {
      const int64_t m = cnt[n];
      free(sp); free(cell); free(cstart); free(cnt);
      const int rc = build_csr(n, m, src, dst, out);
      free(src);
      free(dst);
      return rc;
    }
  }
  return IPGC_GEN_ERR_ARG;  /* not reached */
}

/*
 * 3-D lattice of side^3 nodes (ID = x + side * (y + side * z)), an edge
 * between two nodes whose offset (dx, dy, dz) has dx^2 + dy^2 + dz^2 <= r2;
 * r2 = 6 gives 80 neighbours inside the lattice (fewer at the faces), the
 * degree profile of a regular 3-D finite-element mesh.
 */
int ipgc_gen_lattice3(int32_t side, int32_t r2, ipgc_gen_csr* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (!out || side < 0 || side > 1290 || r2 < 1 || r2 > 16) return IPGC_GEN_ERR_ARG;
  int off[400][3];
  int no = 0;
  const int R = (int)floor(sqrt((double)r2));
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        if (dx * dx + dy * dy + dz * dz > r2) continue;
        /* one of each +-pair: the lexicographically positive (dz, dy, dx) */
        if (dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0)))) continue;
        off[no][0] = dx;
        off[no][1] = dy;
        off[no][2] = dz;
        ++no;
      }
  const int64_t n = (int64_t)side * side * side;
  if (n > INT32_MAX) return IPGC_GEN_ERR_TOO_BIG;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return IPGC_GEN_ERR_OOM;
  for (int pass = 0; pass < 2; ++pass) {
    int32_t* src = NULL;
    int32_t* dst = NULL;
    if (pass == 1) {
      for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
      src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
      dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
      if (!src || !dst) {
        free(src); free(dst); free(cnt);
        return IPGC_GEN_ERR_OOM;
      }
    }
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
      const int64_t x = v % side, y = (v / side) % side, z = v / ((int64_t)side * side);
      int64_t k = 0, w = pass ? cnt[v] : 0;
      for (int o = 0; o < no; ++o) {
        const int64_t X = x + off[o][0], Y = y + off[o][1], Z = z + off[o][2];
        if (X < 0 || Y < 0 || Z < 0 || X >= side || Y >= side || Z >= side) continue;
        if (pass) {
          src[w] = (int32_t)v;
          dst[w] = (int32_t)(X + side * (Y + (int64_t)side * Z));
          ++w;
        }
        ++k;
      }
      if (!pass) cnt[v + 1] = k;
    }
    if (pass == 1) {
      const int64_t m = cnt[n];
      free(cnt);
      const int rc = build_csr((int32_t)n, m, src, dst, out);
      free(src);
      free(dst);
      return rc;
    }
  }
  return IPGC_GEN_ERR_ARG;  /* not reached */
}

/*
 * Hub-heavy graph: m_base uniform pairs over n nodes (an Erdos-Renyi-like
 * base; self-loops and repeats dropped by the CSR build), plus nhubs hubs,
 * hub h (a uniform node) joined to round(max_deg / (h + 1)^alpha) uniform
 * nodes. Every stream is per chunk of 2^16 draws or per hub.
 */
int ipgc_gen_hubs(uint64_t seed, int32_t n, int64_t m_base, int32_t nhubs, int64_t max_deg, double alpha,
            ipgc_gen_csr* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (!out || n < 1 || m_base < 0 || nhubs < 0 || max_deg < 0 || !(alpha >= 0)) return IPGC_GEN_ERR_ARG;
  int64_t* hstart = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nhubs + 1));
  if (!hstart) return IPGC_GEN_ERR_OOM;
  hstart[0] = m_base;
  for (int32_t h = 0; h < nhubs; ++h) {
    int64_t d = (int64_t)llround((double)max_deg / pow((double)(h + 1), alpha));
    if (d > n - 1) d = n - 1;
    hstart[h + 1] = hstart[h] + d;
  }
  const int64_t m = hstart[nhubs];
  int32_t* src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t* dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  if (!src || !dst) {
    free(src); free(dst); free(hstart);
    return IPGC_GEN_ERR_OOM;
  }
  const int64_t chunk = 1 << 16, nch = (m_base + chunk - 1) / chunk;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nch; ++k) {
    rng_t rr;
    rng_seed(&rr, ipgc_gen_derive_seed(seed, (uint64_t)k));
    const int64_t hi = (k + 1) * chunk < m_base ? (k + 1) * chunk : m_base;
    for (int64_t e = k * chunk; e < hi; ++e) {
      src[e] = (int32_t)rng_below(&rr, (uint64_t)n);
      dst[e] = (int32_t)rng_below(&rr, (uint64_t)n);
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t h = 0; h < nhubs; ++h) {
    rng_t rr;
    rng_seed(&rr, ipgc_gen_derive_seed(seed ^ 0x68756273ULL, (uint64_t)h));
    const int32_t hub = (int32_t)rng_below(&rr, (uint64_t)n);
    for (int64_t e = hstart[h]; e < hstart[h + 1]; ++e) {
      src[e] = hub;
      dst[e] = (int32_t)rng_below(&rr, (uint64_t)n);
    }
  }
  free(hstart);
  const int rc = build_csr(n, m, src, dst, out);
  free(src);
  free(dst);
  return rc;
}

void ipgc_gen_free_csr(ipgc_gen_csr* g) {
  if (!g) return;
  free(g->rowptr);
  free(g->col);
  g->rowptr = NULL;
  g->col = NULL;
  g->n = 0;
  g->nnz = 0;
}

/* ------------------------------------------------------------- batches -- */

/*
 * A batch of independent graphs. Graph g draws its node count and parameters
 * from ipgc_gen_derive_seed(seed, g), so each graph depends only on (seed, g) and
 * the batch is the same whatever the number of host threads:
 *   n_g = floor(exp(U(ln nmin, ln(nmax + 1)))) clamped to [nmin, nmax]
 *   even g: Erdos-Renyi with average degree U(deg_lo, deg_hi), m = round(n d / 2)
 *   odd g:  RMAT (a, b, c as given) with scale ceil(log2 n_g), edge factor
 *           rmat_ef (nedges = ef * n_g), endpoints >= n_g redrawn, IDs permuted.
 * Outputs are concatenated: node_off[G+1], edge_off[G+1] (int64 prefix sums),
 * rowptr_cat (graph g's local rowptr of n_g + 1 entries starts at
 * node_off[g] + g) and col_cat (graph g's local neighbour IDs start at
 * edge_off[g]).
 */
int ipgc_gen_batch(uint64_t seed, int32_t num_graphs, int32_t nmin, int32_t nmax, double deg_lo,
             double deg_hi, int32_t rmat_ef, double a, double b, double c, ipgc_gen_batch_t* out) {
  if (out) memset(out, 0, sizeof(*out)); /* no memory on any error */
  if (!out || num_graphs < 0 || nmin < 2 || nmax < nmin || deg_lo < 0 || deg_hi < deg_lo ||
      rmat_ef < 0)
    return IPGC_GEN_ERR_ARG;
  memset(out, 0, sizeof(*out));
  ipgc_gen_csr* gs = (ipgc_gen_csr*)calloc((size_t)(num_graphs > 0 ? num_graphs : 1), sizeof(ipgc_gen_csr));
  if (!gs) return IPGC_GEN_ERR_OOM;
  int failed = IPGC_GEN_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t g = 0; g < num_graphs; ++g) {
    rng_t r;
    uint64_t gseed = ipgc_gen_derive_seed(seed, (uint64_t)g);
    rng_seed(&r, gseed);
    double lo = log((double)nmin), hi = log((double)nmax + 1.0);
    int32_t ng = (int32_t)floor(exp(lo + (hi - lo) * rng_unit(&r)));
    if (ng < nmin) ng = nmin;
    if (ng > nmax) ng = nmax;
    int rc;
    if ((g & 1) == 0) {
      double d = deg_lo + (deg_hi - deg_lo) * rng_unit(&r);
      int64_t m = (int64_t)llround((double)ng * d * 0.5);
      int64_t mmax = (int64_t)ng * (ng - 1) / 2;
      if (m > mmax) m = mmax;
      rc = ipgc_gen_er(rng_u64(&r), ng, m, &gs[g]);
    } else {
      int32_t sc = 0;
      while (((int64_t)1 << sc) < ng) ++sc;
      rc = ipgc_gen_rmat(rng_u64(&r), sc, (int64_t)rmat_ef * ng, a, b, c, ng, 1, &gs[g]);
    }
    if (rc != IPGC_GEN_OK) {
#pragma omp critical
      failed = rc;
    }
  }
  if (failed != IPGC_GEN_OK) {
    for (int32_t g = 0; g < num_graphs; ++g) ipgc_gen_free_csr(&gs[g]);
    free(gs);
    return failed;
  }
  int64_t* node_off = (int64_t*)malloc(((size_t)num_graphs + 1) * sizeof(int64_t));
  int64_t* edge_off = (int64_t*)malloc(((size_t)num_graphs + 1) * sizeof(int64_t));
  if (!node_off || !edge_off) {
    free(node_off);
    free(edge_off);
    for (int32_t g = 0; g < num_graphs; ++g) ipgc_gen_free_csr(&gs[g]);
    free(gs);
    return IPGC_GEN_ERR_OOM;
  }
  node_off[0] = 0;
  edge_off[0] = 0;
  for (int32_t g = 0; g < num_graphs; ++g) {
    node_off[g + 1] = node_off[g] + gs[g].n;
    edge_off[g + 1] = edge_off[g] + gs[g].nnz;
  }
  int64_t nrp = node_off[num_graphs] + num_graphs;
  int64_t ncol = edge_off[num_graphs];
  int32_t* rp = (int32_t*)malloc((size_t)(nrp > 0 ? nrp : 1) * sizeof(int32_t));
  int32_t* cl = (int32_t*)malloc((size_t)(ncol > 0 ? ncol : 1) * sizeof(int32_t));
  if (!rp || !cl) {
    free(rp);
    free(cl);
    free(node_off);
    free(edge_off);
    for (int32_t g = 0; g < num_graphs; ++g) ipgc_gen_free_csr(&gs[g]);
    free(gs);
    return IPGC_GEN_ERR_OOM;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t g = 0; g < num_graphs; ++g) {
    memcpy(rp + node_off[g] + g, gs[g].rowptr, ((size_t)gs[g].n + 1) * sizeof(int32_t));
    if (gs[g].nnz > 0)
      memcpy(cl + edge_off[g], gs[g].col, (size_t)gs[g].nnz * sizeof(int32_t));
    ipgc_gen_free_csr(&gs[g]);
  }
  free(gs);
  out->num_graphs = num_graphs;
  out->node_off = node_off;
  out->edge_off = edge_off;
  out->rowptr_cat = rp;
  out->col_cat = cl;
  return IPGC_GEN_OK;
}

void ipgc_gen_free_batch(ipgc_gen_batch_t* bt) {
  if (!bt) return;
  free(bt->node_off);
  free(bt->edge_off);
  free(bt->rowptr_cat);
  free(bt->col_cat);
  memset(bt, 0, sizeof(*bt));
}

/* ---------------------------------------------------------------- hash -- */

/* FNV-1a (64-bit) over little-endian 32-bit words, used to record inputs. */
uint64_t ipgc_gen_hash_words(const int32_t* p, int64_t count, uint64_t h) {
  if (h == 0) h = 0xcbf29ce484222325ULL;
  for (int64_t i = 0; i < count; ++i) {
    uint32_t w = (uint32_t)p[i];
    for (int k = 0; k < 4; ++k) {
      h ^= (uint64_t)((w >> (8 * k)) & 0xffu);
      h *= 0x100000001b3ULL;
    }
  }
  return h;
}

int ipgc_gen_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
