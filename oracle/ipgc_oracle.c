/*
 * IPGC CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the Iterative Parallel Graph
 * Coloring (IPGC) loop of "A Hybrid Graph Coloring Algorithm for GPUs"
 * (Section II-C), written to decide what the GPU path must output. Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * product library never links, loads or calls it, and this file shares no
 * code with the CUDA sources.
 *
 * Round semantics (fixed and deterministic; the paper's own GPU code reads
 * colours concurrently and so is not):
 *   - Section II-C: every node starts with colour 0 = "uncolored" and every
 *     node starts in the worklist A.
 *   - Step 1 (Section II-C, with the footnote's mex): each active node v gets
 *     the tentative colour T[v] = the smallest c >= 1 that is not the colour
 *     of a neighbour. Colours are read from the snapshot taken at the start of
 *     the round; active neighbours count as uncoloured (0). The footnote's
 *     examples mix 0 in; colour 0 is reserved for "uncolored", so the valid
 *     colours are 1, 2, ...
 *   - Step 2 (Section II-C): an edge whose two active endpoints got the same
 *     tentative colour is a conflict; exactly one endpoint stays in the
 *     worklist. The paper gives no tie rule: the endpoint with the higher
 *     node ID loses. Losing is decided on all tentative colours at once.
 *   - Winners keep T[v] as their final colour and leave the worklist; losers
 *     stay uncoloured and form the next worklist. The loop ends when the
 *     worklist is empty (Section II-C).
 *   - A round is one step 1 plus one step 2; the last, conflict-free round is
 *     counted. The colour count is the largest colour used.
 *
 * Whether a round is run topology-driven or data-driven (Section IV) does not
 * change any of this, so the oracle has no notion of modes.
 *
 * Input: an undirected simple graph as CSR (rowptr[n + 1], col[nnz]), both
 * directions of every edge present, no self-loops. Row order is not assumed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_OOM (-2)

/*
 * Colour the graph. Outputs:
 *   color[n]        final colour of every node (1..K)
 *   *rounds_out     number of rounds
 *   *colors_out     K = max colour (0 when n == 0)
 *   fin_round[n]    optional (may be NULL): the round in which v was finalised
 *   wl_sizes[cap]   optional (may be NULL): |A| at the start of round r is
 *                   stored at wl_sizes[r - 1] for r <= cap
 *   deg_sums[cap]   optional (may be NULL): sum of deg(v) over A, same index
 */
int oracle_color(const int32_t* rowptr, const int32_t* col, int32_t n, int32_t* color,
                 int32_t* rounds_out, int32_t* colors_out, int32_t* fin_round, int64_t* wl_sizes,
                 int64_t* deg_sums, int32_t cap) {
  if (n < 0 || !color || !rounds_out || !colors_out) return ORACLE_ERR_ARG;
  if (n > 0 && (!rowptr || (rowptr[n] > 0 && !col))) return ORACLE_ERR_ARG;
  *rounds_out = 0;
  *colors_out = 0;
  if (n == 0) return ORACLE_OK;

  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t d = rowptr[v + 1] - rowptr[v];
    if (d > maxdeg) maxdeg = d;
  }

  int32_t* A = (int32_t*)malloc((size_t)n * sizeof(int32_t));      /* worklist */
  int32_t* nextA = (int32_t*)malloc((size_t)n * sizeof(int32_t));  /* next worklist */
  int32_t* T = (int32_t*)malloc((size_t)n * sizeof(int32_t));      /* tentative colours */
  char* active = (char*)malloc((size_t)n);                          /* v in A */
  char* lose = (char*)malloc((size_t)n);
  int64_t* seen = (int64_t*)malloc(((size_t)maxdeg + 2) * sizeof(int64_t)); /* colour marks */
  if (!A || !nextA || !T || !active || !lose || !seen) {
    free(A);
    free(nextA);
    free(T);
    free(active);
    free(lose);
    free(seen);
    return ORACLE_ERR_OOM;
  }

  /* Initially every node has colour 0 and is in the worklist. */
  int32_t na = n;
  for (int32_t v = 0; v < n; ++v) {
    color[v] = 0;
    A[v] = v;
    active[v] = 1;
    if (fin_round) fin_round[v] = 0;
  }
  for (int32_t c = 0; c < maxdeg + 2; ++c) seen[c] = -1;
  int64_t stamp = 0;
  int32_t round = 0;

  while (na > 0) {
    round += 1;
    if (wl_sizes && round <= cap) wl_sizes[round - 1] = na;
    if (deg_sums && round <= cap) {
      int64_t s = 0;
      for (int32_t i = 0; i < na; ++i) s += rowptr[A[i] + 1] - rowptr[A[i]];
      deg_sums[round - 1] = s;
    }

    /* Step 1: T[v] = mex over c >= 1 of the neighbours' committed colours.
     * color[] is not written in this loop, so every v sees the same snapshot.
     * T[v] <= deg(v) + 1, so colours above deg(v) + 1 cannot matter. */
    for (int32_t i = 0; i < na; ++i) {
      int32_t v = A[i];
      int32_t deg = rowptr[v + 1] - rowptr[v];
      ++stamp;
      for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
        int32_t c = color[col[k]];
        if (c >= 1 && c <= deg + 1) seen[c] = stamp;
      }
      int32_t t = 1;
      while (seen[t] == stamp) ++t;
      T[v] = t;
    }

    /* Step 2: v loses iff an active neighbour u with a lower ID has the same
     * tentative colour. Uses the T of every active node at once. */
    for (int32_t i = 0; i < na; ++i) {
      int32_t v = A[i];
      char l = 0;
      for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
        int32_t u = col[k];
        if (active[u] && u < v && T[u] == T[v]) {
          l = 1;
          break;
        }
      }
      lose[v] = l;
    }

    /* Winners commit their colour and leave; losers stay uncoloured. */
    int32_t nn = 0;
    for (int32_t i = 0; i < na; ++i) {
      int32_t v = A[i];
      if (lose[v]) {
        nextA[nn++] = v;
      } else {
        color[v] = T[v];
        active[v] = 0;
        if (fin_round) fin_round[v] = round;
        if (T[v] > *colors_out) *colors_out = T[v];
      }
    }
    int32_t* t = A;
    A = nextA;
    nextA = t;
    na = nn;
  }
  *rounds_out = round;

  free(A);
  free(nextA);
  free(T);
  free(active);
  free(lose);
  free(seen);
  return ORACLE_OK;
}

/*
 * The paper's micro-benchmark (Section III): every iteration deactivates the
 * next COUNT node IDs and re-pushes the rest. The text says iteration 0
 * deactivates nodes 0..COUNT-1, so iteration i keeps node v iff
 * v >= COUNT * (i + 1). Returns the number of iterations until the worklist
 * is empty; sizes[i] (optional, up to cap) is |WL| after iteration i.
 */
int64_t oracle_push_iterations(int32_t n, int32_t count, int64_t* sizes, int64_t cap) {
  if (n < 0 || count <= 0) return ORACLE_ERR_ARG;
  int64_t iter = 0;
  int64_t left = n;
  while (left > 0) {
    int64_t keep = 0;
    for (int64_t v = 0; v < n; ++v)
      if (v >= (int64_t)count * (iter + 1)) ++keep;
    if (sizes && iter < cap) sizes[iter] = keep;
    left = keep;
    ++iter;
  }
  return iter;
}

/*
 * Both kernels of the Section III micro-benchmark, run in a Pipe until the
 * worklist is empty, as the paper writes them. mode 0 (Push_WL) pops every
 * worklist entry and pushes it back iff it stays active; mode 1 (Push_NoWL)
 * visits every node of the graph and pushes it iff it is active. A node v
 * stays active in iteration i iff v >= count * (i + 1). After iteration i,
 * sizes[i] = |WL| and sums[i] = the sum of the IDs in WL (optional arrays of
 * cap entries). Returns the number of iterations.
 */
int64_t oracle_push_run(int32_t n, int32_t count, int32_t mode, int64_t* sizes, int64_t* sums,
                        int64_t cap) {
  if (n < 0 || count <= 0 || (mode != 0 && mode != 1)) return ORACLE_ERR_ARG;
  int32_t* wl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!wl || !next) {
    free(wl);
    free(next);
    return ORACLE_ERR_OOM;
  }
  int64_t len = n;  /* WL = graph.nodes */
  for (int32_t v = 0; v < n; ++v) wl[v] = v;
  int64_t iter = 0;
  while (len > 0) {
    const int64_t thr = (int64_t)count * (iter + 1);
    int64_t nlen = 0, sum = 0;
    if (mode == 0) {
      for (int64_t k = 0; k < len; ++k) {
        const int32_t v = wl[k]; /* pop */
        if (v >= thr) {
          next[nlen++] = v; /* push */
          sum += v;
        }
      }
    } else {
      for (int32_t v = 0; v < n; ++v) {
        if (v >= thr) {
          next[nlen++] = v;
          sum += v;
        }
      }
    }
    if (sizes && iter < cap) sizes[iter] = nlen;
    if (sums && iter < cap) sums[iter] = sum;
    int32_t* t = wl;
    wl = next;
    next = t;
    len = nlen;
    ++iter;
  }
  free(wl);
  free(next);
  return iter;
}
