/* tcurve_oracle.h -- CPU oracle for the real scheme of a T-curve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this code; only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py use it.  It shares no code with
 * the CUDA engine.
 *
 * What it computes (Sec. 2, "Fast Isotopy Computation for T-Curves"): the
 * real scheme of the patchworked piecewise-linear curve C(T, sigma), i.e.
 * the isotopy type in RP^2 of the union of segments joining the midpoints
 * of the sign-changing edges of the reflected triangulation T^diamond with
 * antipodal boundary points identified.  It does NOT follow Algorithm 1: it
 * builds the curve itself, walks its components, tells ovals from the
 * pseudoline by the parity of their passages through the line at infinity,
 * and decides nesting by exact ray-parity tests on the two-sheeted sphere
 * covering RP^2.
 *
 * Conventions shared with the engine's C ABI (definitions, not code):
 *   lattice index k(i,j) = j(d+1) - j(j-1)/2 + i for (i,j) in A (Eq. 1);
 *   bit k of the sign words (word k/64, bit k%64) is sigma(i,j); bit 1 means
 *   a negative coefficient, since the coefficient sign is (-1)^sigma (Thm. 1).
 *   Output: canonical nesting-tree code, little-endian uint64 words, value
 *   (1 << nbits) | bits, bits = the root's children encodings in descending
 *   lexicographic order, enc(oval) = '1' . children . '0'.
 */
#ifndef TCURVE_ORACLE_H
#define TCURVE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_D 16

/* Per-instance facts reported beside the code (for the pins in tests/). */
typedef struct {
  int32_t n_ovals;        /* two-sided components                         */
  int32_t n_pseudolines;  /* one-sided components                         */
  int32_t max_depth;      /* deepest nest: 1 for unnested ovals, 0 if none */
  int32_t n_even;         /* ovals inside an even number of ovals (p)     */
  int32_t n_odd;          /* ovals inside an odd number of ovals  (n)     */
  int32_t n_segments;     /* mixed triangles of T^diamond                 */
  int32_t n_crossed;      /* crossed edges of T^diamond                   */
  int32_t n_retries;      /* ray endpoints rejected as non-generic        */
} orc_stats;

/* Error codes (negative). */
#define ORC_OK            0
#define ORC_EINVAL       -1  /* bad degree or arguments                        */
#define ORC_ENOTTRI      -2  /* edges do not form a unimodular triangulation   */
#define ORC_ECURVE       -3  /* a curve vertex without exactly two segments    */
#define ORC_ETOPOLOGY    -4  /* pseudoline count or laminarity violated        */
#define ORC_EOVERFLOW    -5  /* code does not fit the given words              */
#define ORC_EGENERIC     -6  /* no generic ray endpoint found                  */

/* Number of uint64 words of a code: ceil((2*nmax+1)/64) with nmax = M for
 * even d and M-1 for odd d, M = (d-1)(d-2)/2 + 1 (Harnack's bound). */
int orc_code_words(int d);

/* Triangles of T from its edge list: (n_edges x 4) int32 rows (i1,j1,i2,j2).
 * Writes n_tri x 6 int32 rows (i1,j1,i2,j2,i3,j3), counter-clockwise, and
 * returns n_tri (= d*d) or a negative error. */
int orc_triangles_from_edges(int d, int n_edges, const int32_t *edges,
                             int32_t *tri_out, int max_tri);

/* Real scheme of one (T, sigma).  tri: d*d rows from
 * orc_triangles_from_edges.  sigma: ceil(|A|/64) words.  code: code_words
 * words.  stats may be NULL.  Returns ORC_OK or a negative error. */
int orc_real_scheme(int d, const int32_t *tri, const uint64_t *sigma,
                    uint64_t *code, int code_words, orc_stats *stats);

/* Many instances on n_threads POSIX threads.  sigmas: n x sign_words,
 * codes: n x code_words, status: n entries (may be NULL), stats: n entries
 * (may be NULL).  Returns the number of instances that failed. */
int64_t orc_real_schemes_batch(int d, const int32_t *tri, int sign_words,
                               const uint64_t *sigmas, int64_t n,
                               uint64_t *codes, int code_words,
                               int32_t *status, orc_stats *stats,
                               int n_threads);

#ifdef __cplusplus
}
#endif
#endif
