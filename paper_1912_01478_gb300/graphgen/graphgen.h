/*
 * Seeded synthetic graph generators (host C). Inputs only: no colouring logic.
 * Every function returns GG_OK (0) or a negative GG_ERR_* code and never
 * aborts. Arrays in gg_csr / gg_batch_t are malloc()ed by this library and
 * owned by the caller until gg_free_csr / gg_free_batch.
 */
#ifndef GRAPHGEN_H
#define GRAPHGEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { GG_OK = 0, GG_ERR_ARG = -1, GG_ERR_OOM = -2, GG_ERR_TOO_BIG = -3 };

typedef struct {
  int32_t n;       /* nodes */
  int64_t nnz;     /* directed CSR entries (2 x undirected edges) */
  int32_t* rowptr; /* int32[n + 1] */
  int32_t* col;    /* int32[nnz], each row sorted ascending */
} gg_csr;

typedef struct {
  int32_t num_graphs;
  int64_t* node_off;   /* int64[G + 1] */
  int64_t* edge_off;   /* int64[G + 1] */
  int32_t* rowptr_cat; /* graph g's local rowptr (n_g + 1 entries) at node_off[g] + g */
  int32_t* col_cat;    /* graph g's local column IDs at edge_off[g] */
} gg_batch_t;

uint64_t gg_derive_seed(uint64_t seed, uint64_t index);
int gg_from_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, gg_csr* out);
int gg_er(uint64_t seed, int32_t n, int64_t m, gg_csr* out);
int gg_rmat(uint64_t seed, int32_t scale, int64_t nedges, double a, double b, double c,
            int32_t n_limit, int32_t permute, gg_csr* out);
int gg_road(uint64_t seed, int32_t side, double p_delete, double frac_long, gg_csr* out);
int gg_rgg(uint64_t seed, int32_t n, int32_t dim, double avg_degree, gg_csr* out);
int gg_lattice3(int32_t side, int32_t r2, gg_csr* out);
int gg_hubs(uint64_t seed, int32_t n, int64_t m_base, int32_t nhubs, int64_t max_deg, double alpha,
            gg_csr* out);
int gg_batch(uint64_t seed, int32_t num_graphs, int32_t nmin, int32_t nmax, double deg_lo,
             double deg_hi, int32_t rmat_ef, double a, double b, double c, gg_batch_t* out);
void gg_free_csr(gg_csr* g);
void gg_free_batch(gg_batch_t* b);
uint64_t gg_hash_words(const int32_t* p, int64_t count, uint64_t h);
int gg_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
