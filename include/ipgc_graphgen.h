/*
 * ipgc_graphgen.h -- C ABI of libgraphgen.so: the seeded synthetic graph
 * generators and the CSR symmetriser that make the colouring's inputs.
 *
 * The colouring problem is stated on an undirected graph G = (V, E)
 * (Section II-A), and the paper removes self-loops and multi-edges from its
 * inputs before colouring them (Section V). Every graph returned here is in
 * that form, as the CSR that ipgc_color takes (include/ipgc.h, "Graph
 * input"):
 *   - undirected: both directed entries of every edge are present;
 *   - no self-loop, no duplicate entry, every row sorted ascending;
 *   - int32 rowptr[n + 1] (rowptr[0] = 0, rowptr[n] = nnz) and int32 col[nnz].
 * The paper's own inputs (UFL/SuiteSparse matrices, Table I) are not
 * available here; these generators make seeded stand-ins with the shapes of
 * Table I (sizes, degree distribution, ID locality).
 *
 * This library holds no colouring arithmetic: it only makes inputs. Both the
 * GPU path and the CPU oracle's tests consume its byte-identical output.
 *
 * Random numbers: xoshiro256** seeded through splitmix64 (both from their
 * published definitions). The output depends only on the arguments: it is
 * the same for any number of host threads and on x86-64 and aarch64 hosts.
 *
 * Conventions for every entry point:
 *   - returns IPGC_GEN_OK (0) or a negative IPGC_GEN_ERR_* code; never
 *     aborts, prints or throws; on error *out holds no memory;
 *   - every pointer is HOST memory; the arrays in ipgc_gen_csr and
 *     ipgc_gen_batch_t are malloc()ed by the library and owned by the caller
 *     until ipgc_gen_free_csr / ipgc_gen_free_batch;
 *   - the generators run on the host's OpenMP threads.
 */
#ifndef IPGC_GRAPHGEN_H
#define IPGC_GRAPHGEN_H

#include <stdint.h>

#if defined(__GNUC__)
#define IPGC_GEN_API __attribute__((visibility("default")))
#else
#define IPGC_GEN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define IPGC_GEN_OK 0
#define IPGC_GEN_ERR_ARG (-1)     /* an argument is out of range */
#define IPGC_GEN_ERR_OOM (-2)     /* host allocation failed */
#define IPGC_GEN_ERR_TOO_BIG (-3) /* the graph would have 2^31 or more CSR entries */

/* One graph. */
typedef struct ipgc_gen_csr {
  int32_t n;       /* nodes */
  int64_t nnz;     /* directed CSR entries (2 x undirected edges) */
  int32_t* rowptr; /* int32[n + 1] */
  int32_t* col;    /* int32[nnz], each row strictly ascending */
} ipgc_gen_csr;

/* Many graphs, concatenated in the layout ipgc_color_batched takes. */
typedef struct ipgc_gen_batch_t {
  int32_t num_graphs;  /* G */
  int64_t* node_off;   /* int64[G + 1]: graph g has nodes [node_off[g], node_off[g + 1]) */
  int64_t* edge_off;   /* int64[G + 1]: graph g's entries are col_cat[edge_off[g] ..) */
  int32_t* rowptr_cat; /* graph g's local rowptr (n_g + 1 entries) at node_off[g] + g */
  int32_t* col_cat;    /* graph g's local neighbour IDs (0 .. n_g - 1) at edge_off[g] */
} ipgc_gen_batch_t;

/*
 * The symmetriser: the CSR of the undirected graph on n nodes with the m
 * pairs (src[e], dst[e]) as edges, each pair entered in both directions,
 * self-loops dropped, duplicates merged, rows sorted (Section V's
 * preprocessing). src, dst: host int32[m], every value in [0, n).
 * IPGC_GEN_ERR_ARG for n < 0, m < 0 or a value out of range.
 */
IPGC_GEN_API int ipgc_gen_from_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                     ipgc_gen_csr* out);

/*
 * Erdos-Renyi G(n, m): exactly m distinct undirected edges between uniformly
 * drawn node pairs (self-loops and repeats redrawn); m <= n (n - 1) / 2.
 * The Erdos-Renyi workload is n = 10,000, m = 40,000 (average degree 8), seed 1.
 */
IPGC_GEN_API int ipgc_gen_er(uint64_t seed, int32_t n, int64_t m, ipgc_gen_csr* out);

/*
 * RMAT without noise, standing in for the paper's Kronecker and power-law
 * graphs (Table I: kron_g500-logn21, soc-LiveJournal1, hollywood-2009): nedges
 * directed draws over a 2^scale square, quadrant probabilities a, b, c and
 * d = 1 - a - b - c at every bit, then symmetrised and deduplicated. With
 * n_limit in (0, 2^scale) the graph has n_limit nodes and a draw with an
 * endpoint >= n_limit is redrawn whole; permute != 0 relabels the IDs by a
 * Fisher-Yates permutation. The RMAT workload is scale 22, nedges = 16 x 2^22,
 * a, b, c = 0.57, 0.19, 0.19, permuted, seed 2. scale in [0, 30].
 */
IPGC_GEN_API int ipgc_gen_rmat(uint64_t seed, int32_t scale, int64_t nedges, double a, double b,
                               double c, int32_t n_limit, int32_t permute, ipgc_gen_csr* out);

/*
 * Road-network-like graph, standing in for europe_osm (Table I): a side x
 * side 4-neighbour grid with row-major IDs (not permuted), every grid edge
 * deleted with probability p_delete, then round(frac_long x retained)
 * long-range edges with uniform endpoints added. The road workload is
 * side = 4096, p_delete = 0.3, frac_long = 0.01, seed 3. side <= 46340.
 */
IPGC_GEN_API int ipgc_gen_road(uint64_t seed, int32_t side, double p_delete, double frac_long,
                               ipgc_gen_csr* out);

/*
 * Random geometric graph, standing in for rgg_n_2_24_s0 and the finite
 * element meshes of Table I: n points uniform in the unit square (dim 2) or
 * cube (dim 3), an edge between points closer than the radius that gives
 * mean degree avg_degree away from the border; IDs in grid-cell order.
 */
IPGC_GEN_API int ipgc_gen_rgg(uint64_t seed, int32_t n, int32_t dim, double avg_degree,
                              ipgc_gen_csr* out);

/*
 * side^3 lattice with an edge between nodes at squared distance <= r2
 * (r2 = 6: 80 neighbours inside), standing in for Queen_4147 (Table I).
 */
IPGC_GEN_API int ipgc_gen_lattice3(int32_t side, int32_t r2, ipgc_gen_csr* out);

/*
 * Hub-heavy graph, standing in for circuit5M (Table I): m_base uniform pairs
 * on n nodes plus nhubs hubs, hub h of degree about max_deg / (h + 1)^alpha
 * with uniform neighbours.
 */
IPGC_GEN_API int ipgc_gen_hubs(uint64_t seed, int32_t n, int64_t m_base, int32_t nhubs,
                               int64_t max_deg, double alpha, ipgc_gen_csr* out);

/*
 * A batch of independent graphs for the batched and served forms. Graph g
 * depends only on (seed, g): n_g log-uniform in [nmin, nmax]; even g
 * Erdos-Renyi with average degree uniform in [deg_lo, deg_hi]; odd g RMAT
 * (a, b, c) with scale ceil(log2 n_g), rmat_ef x n_g draws, endpoints >= n_g
 * redrawn, IDs permuted. The batched workload is 4096 graphs in [100, 200000],
 * degrees in [4, 32], rmat_ef = 8, a, b, c = 0.57, 0.19, 0.19, seed 4.
 * nmin >= 2.
 */
IPGC_GEN_API int ipgc_gen_batch(uint64_t seed, int32_t num_graphs, int32_t nmin, int32_t nmax,
                                double deg_lo, double deg_hi, int32_t rmat_ef, double a, double b,
                                double c, ipgc_gen_batch_t* out);

/* Release what a generator returned (NULL or an already-freed record: no-op). */
IPGC_GEN_API void ipgc_gen_free_csr(ipgc_gen_csr* g);
IPGC_GEN_API void ipgc_gen_free_batch(ipgc_gen_batch_t* b);

/*
 * FNV-1a (64-bit) over `count` little-endian int32 words, continuing from h
 * (0 = the FNV offset basis): the recorded hash of a generated input is
 * ipgc_gen_hash_words(col, nnz, ipgc_gen_hash_words(rowptr, n + 1, 0)).
 */
IPGC_GEN_API uint64_t ipgc_gen_hash_words(const int32_t* p, int64_t count, uint64_t h);

/* The seed of the index-th sub-stream of `seed` (per chunk or per graph). */
IPGC_GEN_API uint64_t ipgc_gen_derive_seed(uint64_t seed, uint64_t index);

/* Host threads the generators use (OpenMP), 1 without OpenMP. */
IPGC_GEN_API int ipgc_gen_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif /* IPGC_GRAPHGEN_H */
