/* tcurve_oracle.c -- plain, slow, exact CPU oracle for the real scheme of a
 * T-curve.  TEST INFRASTRUCTURE ONLY (see tcurve_oracle.h): the engine never
 * includes, links or calls this file.
 *
 * Steps, in the order of the definition in Sec. 2:
 *   1. reflect T into the four quadrants to get T^diamond on the diamond
 *      A^diamond = {|x|+|y| <= d} and extend sigma by Eq. 2;
 *   2. an edge is crossed when its end points have distinct signs; every
 *      triangle with a crossed edge has exactly two, and the curve
 *      C(T, sigma) contains the segment joining their midpoints;
 *   3. the diamond with antipodal boundary points identified is RP^2, so a
 *      crossed boundary edge e and its antipode -e are one curve vertex;
 *      walking segment to segment gives the components, and a component
 *      that passes through the boundary an odd number of times is one-sided
 *      (a pseudoline), otherwise it is an oval;
 *   4. nesting: RP^2 is covered by the sphere made of two copies D_U, D_L of
 *      the diamond glued by y_U ~ (-y)_L on the boundary.  Lift an oval B
 *      to one closed curve B~ by switching sheet at every boundary passage.
 *      A point P lies in the disk bounded by B iff its two lifts P_U and
 *      P_L are separated by B~, i.e. iff the path [P, x] in D_U followed by
 *      [-x, P] in D_L (x on the boundary) crosses B~ an odd number of times;
 *   5. the containment relation of the ovals is a forest; the real scheme
 *      is that rooted tree, printed as the canonical code of the header.
 * All coordinates are integers scaled by S = 4*Q, Q prime, so that edge
 * midpoints, segment midpoints and the ray end points are exact; a ray end
 * point that touches the curve non-generically is replaced by the next one.
 */
#include "tcurve_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define Q 1009
#define S (4 * Q)

static int lattice_index(int d, int i, int j) {
  return j * (d + 1) - j * (j - 1) / 2 + i;
}

static int harnack_M(int d) { return (d - 1) * (d - 2) / 2 + 1; }

int orc_code_words(int d) {
  int nmax = (d % 2 == 0) ? harnack_M(d) : harnack_M(d) - 1;
  return (2 * nmax + 1 + 63) / 64;
}

static int64_t orient(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                      int64_t cx, int64_t cy) {
  return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

/* ------------------------------------------------------------------------ */
/* triangles of T from its edge list                                        */
/* ------------------------------------------------------------------------ */

int orc_triangles_from_edges(int d, int n_edges, const int32_t *edges,
                             int32_t *tri_out, int max_tri) {
  if (d < 1 || d > ORC_MAX_D || n_edges < 0 || !edges || !tri_out)
    return ORC_EINVAL;
  int np = (d + 1) * (d + 2) / 2;
  unsigned char *adj = (unsigned char *)calloc((size_t)np * np, 1);
  int *pi = (int *)malloc(sizeof(int) * np), *pj = (int *)malloc(sizeof(int) * np);
  int rc = 0, nt = 0;
  for (int j = 0; j <= d; j++)
    for (int i = 0; i + j <= d; i++) {
      pi[lattice_index(d, i, j)] = i;
      pj[lattice_index(d, i, j)] = j;
    }
  for (int e = 0; e < n_edges; e++) {
    int i1 = edges[4 * e], j1 = edges[4 * e + 1], i2 = edges[4 * e + 2], j2 = edges[4 * e + 3];
    if (i1 < 0 || j1 < 0 || i1 + j1 > d || i2 < 0 || j2 < 0 || i2 + j2 > d) { rc = ORC_ENOTTRI; goto out; }
    int a = lattice_index(d, i1, j1), b = lattice_index(d, i2, j2);
    if (a == b || adj[a * np + b]) { rc = ORC_ENOTTRI; goto out; }
    adj[a * np + b] = adj[b * np + a] = 1;
  }
  /* a triangle is a 3-clique of edges of area 1/2 */
  for (int a = 0; a < np; a++)
    for (int b = a + 1; b < np; b++) {
      if (!adj[a * np + b]) continue;
      for (int c = b + 1; c < np; c++) {
        if (!adj[a * np + c] || !adj[b * np + c]) continue;
        int64_t o = orient(pi[a], pj[a], pi[b], pj[b], pi[c], pj[c]);
        if (o != 1 && o != -1) continue;
        if (nt >= max_tri) { rc = ORC_ENOTTRI; goto out; }
        int p[3] = {a, b, c};
        if (o < 0) { p[1] = c; p[2] = b; }
        for (int k = 0; k < 3; k++) {
          tri_out[6 * nt + 2 * k] = pi[p[k]];
          tri_out[6 * nt + 2 * k + 1] = pj[p[k]];
        }
        nt++;
      }
    }
  if (nt != d * d) { rc = ORC_ENOTTRI; goto out; }
  /* every point is a vertex; edges on the boundary of d*Delta_2 lie in one
   * triangle, all other edges in two */
  {
    int *cnt = (int *)calloc((size_t)np * np, sizeof(int));
    int *used = (int *)calloc((size_t)np, sizeof(int));
    for (int t = 0; t < nt; t++) {
      int v[3];
      for (int k = 0; k < 3; k++) v[k] = lattice_index(d, tri_out[6 * t + 2 * k], tri_out[6 * t + 2 * k + 1]);
      for (int k = 0; k < 3; k++) {
        used[v[k]] = 1;
        int a = v[k], b = v[(k + 1) % 3];
        cnt[a * np + b]++;
        cnt[b * np + a]++;
      }
    }
    for (int a = 0; a < np && !rc; a++) {
      if (!used[a]) rc = ORC_ENOTTRI;
      for (int b = a + 1; b < np && !rc; b++) {
        if (!adj[a * np + b]) continue;
        int on_side = (pi[a] == 0 && pi[b] == 0) || (pj[a] == 0 && pj[b] == 0) ||
                      (pi[a] + pj[a] == d && pi[b] + pj[b] == d);
        if (cnt[a * np + b] != (on_side ? 1 : 2)) rc = ORC_ENOTTRI;
      }
    }
    free(cnt);
    free(used);
  }
out:
  free(adj);
  free(pi);
  free(pj);
  return rc ? rc : nt;
}

/* ------------------------------------------------------------------------ */
/* the diamond complex and the curve                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d, nv, nt, ne;
  int *vid;             /* (x+d)*(2d+1) + (y+d) -> vertex id, or -1 */
  int *vx, *vy, *vs;    /* coordinates and sign of each vertex      */
  int *tv;              /* nt x 3 vertex ids                        */
  int *te;              /* nt x 3 edge ids: (v0v1, v1v2, v2v0)      */
  int *ea, *eb;         /* edge end points                          */
  int *et0, *et1;       /* incident triangles (-1 if none)          */
  int *ebd;             /* 1 if both end points lie on the boundary */
  int *anti;            /* antipodal partner of a boundary edge     */
  int *hkey, *hval, hsize;
} cx_t;

static int vid_of(const cx_t *c, int x, int y) {
  return c->vid[(x + c->d) * (2 * c->d + 1) + (y + c->d)];
}

static int edge_find(cx_t *c, int a, int b, int create) {
  if (a > b) { int t = a; a = b; b = t; }
  int key = a * c->nv + b;
  unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(c->hsize - 1);
  for (;;) {
    if (c->hkey[h] == key) return c->hval[h];
    if (c->hkey[h] < 0) {
      if (!create) return -1;
      int e = c->ne++;
      c->hkey[h] = key;
      c->hval[h] = e;
      c->ea[e] = a;
      c->eb[e] = b;
      c->et0[e] = c->et1[e] = -1;
      return e;
    }
    h = (h + 1) & (unsigned)(c->hsize - 1);
  }
}

static void cx_free(cx_t *c) {
  free(c->vid); free(c->vx); free(c->vy); free(c->vs);
  free(c->tv); free(c->te); free(c->ea); free(c->eb);
  free(c->et0); free(c->et1); free(c->ebd); free(c->anti);
  free(c->hkey); free(c->hval);
}

/* Step 1: T^diamond and the signs of Eq. 2. */
static int cx_build(cx_t *c, int d, const int32_t *tri, const uint64_t *sigma) {
  memset(c, 0, sizeof(*c));
  c->d = d;
  int side = 2 * d + 1;
  int maxv = side * side, maxt = 4 * d * d, maxe = 3 * maxt;
  c->vid = (int *)malloc(sizeof(int) * maxv);
  c->vx = (int *)malloc(sizeof(int) * maxv);
  c->vy = (int *)malloc(sizeof(int) * maxv);
  c->vs = (int *)malloc(sizeof(int) * maxv);
  c->tv = (int *)malloc(sizeof(int) * 3 * maxt);
  c->te = (int *)malloc(sizeof(int) * 3 * maxt);
  c->ea = (int *)malloc(sizeof(int) * maxe);
  c->eb = (int *)malloc(sizeof(int) * maxe);
  c->et0 = (int *)malloc(sizeof(int) * maxe);
  c->et1 = (int *)malloc(sizeof(int) * maxe);
  c->ebd = (int *)malloc(sizeof(int) * maxe);
  c->anti = (int *)malloc(sizeof(int) * maxe);
  c->hsize = 1;
  while (c->hsize < 4 * maxe) c->hsize <<= 1;
  c->hkey = (int *)malloc(sizeof(int) * c->hsize);
  c->hval = (int *)malloc(sizeof(int) * c->hsize);
  for (int h = 0; h < c->hsize; h++) c->hkey[h] = -1;
  for (int k = 0; k < maxv; k++) c->vid[k] = -1;

  for (int y = -d; y <= d; y++)
    for (int x = -d; x <= d; x++) {
      int i = x < 0 ? -x : x, j = y < 0 ? -y : y;
      if (i + j > d) continue;
      int v = c->nv++;
      c->vid[(x + d) * side + (y + d)] = v;
      c->vx[v] = x;
      c->vy[v] = y;
      int k = lattice_index(d, i, j);
      int s = (int)((sigma[k >> 6] >> (k & 63)) & 1u);
      /* Eq. 2: sigma(-i,j) = sigma + i, sigma(i,-j) = sigma + j (mod 2) */
      if (x < 0) s ^= (i & 1);
      if (y < 0) s ^= (j & 1);
      c->vs[v] = s;
    }

  static const int qsx[4] = {1, -1, -1, 1}, qsy[4] = {1, 1, -1, -1};
  for (int q = 0; q < 4; q++)
    for (int t = 0; t < d * d; t++) {
      int T = c->nt++;
      for (int k = 0; k < 3; k++)
        c->tv[3 * T + k] = vid_of(c, qsx[q] * tri[6 * t + 2 * k], qsy[q] * tri[6 * t + 2 * k + 1]);
      for (int k = 0; k < 3; k++) {
        int e = edge_find(c, c->tv[3 * T + k], c->tv[3 * T + (k + 1) % 3], 1);
        c->te[3 * T + k] = e;
        if (c->et0[e] < 0) c->et0[e] = T;
        else if (c->et1[e] < 0) c->et1[e] = T;
        else return ORC_ENOTTRI;
      }
    }
  for (int e = 0; e < c->ne; e++) {
    int a = c->ea[e], b = c->eb[e];
    int ba = abs(c->vx[a]) + abs(c->vy[a]) == d, bb = abs(c->vx[b]) + abs(c->vy[b]) == d;
    c->ebd[e] = ba && bb;
    c->anti[e] = -1;
  }
  for (int e = 0; e < c->ne; e++) {
    if (!c->ebd[e]) {
      if (c->et1[e] < 0) return ORC_ENOTTRI;
      continue;
    }
    if (c->et1[e] >= 0) return ORC_ENOTTRI;
    int a = c->ea[e], b = c->eb[e];
    int f = edge_find(c, vid_of(c, -c->vx[a], -c->vy[a]), vid_of(c, -c->vx[b], -c->vy[b]), 0);
    if (f < 0) return ORC_ENOTTRI;
    c->anti[e] = f;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* components of the curve                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t x0, y0, x1, y1; /* scaled end points */
  int sheet;              /* 0 = D_U, 1 = D_L in the lift of its component */
} seg_t;

typedef struct {
  int first, count; /* range in the segment array */
  int jumps;        /* boundary passages          */
  int64_t px, py;   /* test point: midpoint of the first segment */
} comp_t;

static int crossed(const cx_t *c, int e) { return c->vs[c->ea[e]] != c->vs[c->eb[e]]; }

static void edge_mid(const cx_t *c, int e, int64_t *x, int64_t *y) {
  /* (a+b)/2 in units of 1/S */
  *x = (int64_t)(c->vx[c->ea[e]] + c->vx[c->eb[e]]) * (S / 2);
  *y = (int64_t)(c->vy[c->ea[e]] + c->vy[c->eb[e]]) * (S / 2);
}

/* the crossed edge of triangle t other than e_in, or -1 */
static int other_crossed(const cx_t *c, int t, int e_in) {
  int found = -1, n = 0;
  for (int k = 0; k < 3; k++) {
    int e = c->te[3 * t + k];
    if (!crossed(c, e)) continue;
    n++;
    if (e != e_in) found = e;
  }
  return n == 2 ? found : -1;
}

/* Step 3: walk every component once. */
static int walk(const cx_t *c, seg_t *segs, int *nseg, comp_t *comps, int *ncomp) {
  char *seen = (char *)calloc((size_t)c->nt, 1);
  int ns = 0, nc = 0, rc = ORC_OK;
  for (int t0 = 0; t0 < c->nt && rc == ORC_OK; t0++) {
    if (seen[t0]) continue;
    int ea = -1, eb = -1;
    for (int k = 0; k < 3; k++) {
      int e = c->te[3 * t0 + k];
      if (!crossed(c, e)) continue;
      if (ea < 0) ea = e; else eb = e;
    }
    if (ea < 0) continue; /* monochromatic triangle: no segment */
    if (eb < 0) { rc = ORC_ECURVE; break; }
    comp_t *C = &comps[nc++];
    C->first = ns;
    C->jumps = 0;
    int t = t0, e_in = ea, e_out = eb, sheet = 0, steps = 0;
    for (;;) {
      if (seen[t] || ++steps > c->nt) { rc = ORC_ECURVE; break; }
      seen[t] = 1;
      seg_t *sg = &segs[ns++];
      edge_mid(c, e_in, &sg->x0, &sg->y0);
      edge_mid(c, e_out, &sg->x1, &sg->y1);
      sg->sheet = sheet;
      int e = e_out, tn;
      if (c->ebd[e]) {
        /* the midpoint of e is identified with that of -e: jump across */
        C->jumps++;
        sheet ^= 1;
        e = c->anti[e];
        if (!crossed(c, e)) { rc = ORC_ECURVE; break; }
        tn = c->et0[e];
      } else {
        tn = c->et0[e] == t ? c->et1[e] : c->et0[e];
      }
      if (tn == t0 && e == ea) break; /* closed */
      int nxt = other_crossed(c, tn, e);
      if (nxt < 0) { rc = ORC_ECURVE; break; }
      t = tn;
      e_in = e;
      e_out = nxt;
    }
    C->count = ns - C->first;
    C->px = (segs[C->first].x0 + segs[C->first].x1) / 2;
    C->py = (segs[C->first].y0 + segs[C->first].y1) / 2;
  }
  free(seen);
  *nseg = ns;
  *ncomp = nc;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* nesting by ray parity on the sphere cover                                */
/* ------------------------------------------------------------------------ */

/* c lies in the bounding box of [a,b] (used only when a, b, c are collinear) */
static int in_box(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy) {
  return (cx >= (ax < bx ? ax : bx)) && (cx <= (ax < bx ? bx : ax)) &&
         (cy >= (ay < by ? ay : by)) && (cy <= (ay < by ? by : ay));
}

/* 1 if [p1,p2] properly crosses [q1,q2], 0 if they are disjoint, -1 if an
 * end point of one lies on the other (a non-generic ray). */
static int seg_cross(int64_t p1x, int64_t p1y, int64_t p2x, int64_t p2y,
                     int64_t q1x, int64_t q1y, int64_t q2x, int64_t q2y) {
  int64_t o1 = orient(p1x, p1y, p2x, p2y, q1x, q1y);
  int64_t o2 = orient(p1x, p1y, p2x, p2y, q2x, q2y);
  int64_t o3 = orient(q1x, q1y, q2x, q2y, p1x, p1y);
  int64_t o4 = orient(q1x, q1y, q2x, q2y, p2x, p2y);
  if ((o1 == 0 && in_box(p1x, p1y, p2x, p2y, q1x, q1y)) ||
      (o2 == 0 && in_box(p1x, p1y, p2x, p2y, q2x, q2y)) ||
      (o3 == 0 && in_box(q1x, q1y, q2x, q2y, p1x, p1y)) ||
      (o4 == 0 && in_box(q1x, q1y, q2x, q2y, p2x, p2y)))
    return -1;
  if (o1 == 0 || o2 == 0 || o3 == 0 || o4 == 0) return 0;
  return ((o1 > 0) != (o2 > 0)) && ((o3 > 0) != (o4 > 0));
}

/* m-th candidate ray end point on the boundary |X|+|Y| = d*S. */
static void ray_end(int d, int m, int64_t *x, int64_t *y) {
  int64_t L = (int64_t)d * S;
  int64_t t = 1 + ((int64_t)m * 104729 + 13) % (L - 1);
  if (t % Q == 0) t += 1;
  switch (m & 3) {
    case 0: *x = L - t; *y = t; break;
    case 1: *x = -t; *y = L - t; break;
    case 2: *x = -L + t; *y = -t; break;
    default: *x = t; *y = -L + t; break;
  }
}

/* 1 if P lies in the disk bounded by oval B, 0 if not, <0 on failure. */
static int inside(int d, int64_t px, int64_t py, const seg_t *segs, const comp_t *B, int *retries) {
  for (int m = 0; m < 4096; m++) {
    int64_t x, y;
    ray_end(d, m, &x, &y);
    int count = 0, bad = 0;
    for (int s = B->first; s < B->first + B->count && !bad; s++) {
      const seg_t *g = &segs[s];
      int r = g->sheet == 0 ? seg_cross(px, py, x, y, g->x0, g->y0, g->x1, g->y1)
                            : seg_cross(-x, -y, px, py, g->x0, g->y0, g->x1, g->y1);
      if (r < 0) bad = 1; else count += r;
    }
    if (!bad) return count & 1;
    (*retries)++;
  }
  return ORC_EGENERIC;
}

/* ------------------------------------------------------------------------ */
/* canonical code                                                           */
/* ------------------------------------------------------------------------ */

static int cmp_desc(const void *a, const void *b) {
  return strcmp(*(char *const *)b, *(char *const *)a);
}

/* enc(oval) = '1' . (children encodings, descending) . '0' */
static char *encode_children(int parent, int n, const int *par, char **enc) {
  int k = 0;
  size_t len = 0;
  char **kids = (char **)malloc(sizeof(char *) * (n + 1));
  for (int c = 0; c < n; c++)
    if (par[c] == parent) { kids[k++] = enc[c]; len += strlen(enc[c]); }
  qsort(kids, (size_t)k, sizeof(char *), cmp_desc);
  char *out = (char *)malloc(len + 1);
  out[0] = 0;
  size_t pos = 0;
  for (int c = 0; c < k; c++) {
    size_t l = strlen(kids[c]);
    memcpy(out + pos, kids[c], l);
    pos += l;
  }
  out[pos] = 0;
  free(kids);
  return out;
}

int orc_real_scheme(int d, const int32_t *tri, const uint64_t *sigma,
                    uint64_t *code, int code_words, orc_stats *st) {
  if (d < 1 || d > ORC_MAX_D || !tri || !sigma || !code || code_words < 1) return ORC_EINVAL;
  cx_t c;
  int rc = cx_build(&c, d, tri, sigma);
  seg_t *segs = NULL;
  comp_t *comps = NULL;
  int ns = 0, nc = 0, retries = 0;
  int *oval = NULL, *par = NULL, *depth = NULL;
  char *in = NULL, **enc = NULL;
  int no = 0;
  if (rc) goto out;
  segs = (seg_t *)malloc(sizeof(seg_t) * (c.nt + 1));
  comps = (comp_t *)malloc(sizeof(comp_t) * (c.nt + 1));
  rc = walk(&c, segs, &ns, comps, &nc);
  if (rc) goto out;

  /* one-sided components: an odd number of boundary passages */
  int npseudo = 0, jcomp = -1;
  oval = (int *)malloc(sizeof(int) * (nc + 1));
  for (int k = 0; k < nc; k++) {
    if (comps[k].jumps & 1) { npseudo++; jcomp = k; }
    else oval[no++] = k;
  }
  if (npseudo != (d & 1)) { rc = ORC_ETOPOLOGY; goto out; }

  /* in[a*no+b] = oval a lies in the disk of oval b */
  in = (char *)calloc((size_t)no * no + 1, 1);
  for (int a = 0; a < no; a++)
    for (int b = 0; b < no; b++) {
      if (a == b) continue;
      int r = inside(d, comps[oval[a]].px, comps[oval[a]].py, segs, &comps[oval[b]], &retries);
      if (r < 0) { rc = r; goto out; }
      in[a * no + b] = (char)r;
    }
  if (jcomp >= 0)
    for (int b = 0; b < no; b++) {
      int r = inside(d, comps[jcomp].px, comps[jcomp].py, segs, &comps[oval[b]], &retries);
      if (r < 0) { rc = r; goto out; }
      if (r) { rc = ORC_ETOPOLOGY; goto out; } /* a pseudoline bounds no disk */
    }
  /* containment must be a strict partial order whose up-sets are chains */
  for (int a = 0; a < no; a++)
    for (int b = 0; b < no; b++) {
      if (!in[a * no + b]) continue;
      if (in[b * no + a]) { rc = ORC_ETOPOLOGY; goto out; }
      for (int e = 0; e < no; e++) {
        if (in[b * no + e] && !in[a * no + e]) { rc = ORC_ETOPOLOGY; goto out; }
        if (e != b && in[a * no + e] && !in[b * no + e] && !in[e * no + b]) { rc = ORC_ETOPOLOGY; goto out; }
      }
    }
  par = (int *)malloc(sizeof(int) * (no + 1));
  depth = (int *)malloc(sizeof(int) * (no + 1));
  int maxd = -1, peven = 0, nodd = 0;
  for (int a = 0; a < no; a++) {
    depth[a] = 0;
    for (int b = 0; b < no; b++) depth[a] += in[a * no + b];
    if (depth[a] > maxd) maxd = depth[a];
    if (depth[a] & 1) nodd++; else peven++;
  }
  for (int a = 0; a < no; a++) {
    par[a] = -1;
    for (int b = 0; b < no; b++)
      if (in[a * no + b] && depth[b] == depth[a] - 1) par[a] = b;
  }
  /* encodings from the deepest ovals up */
  enc = (char **)calloc((size_t)no + 1, sizeof(char *));
  for (int lev = maxd; lev >= 0; lev--)
    for (int a = 0; a < no; a++) {
      if (depth[a] != lev) continue;
      char *inner = encode_children(a, no, par, enc);
      size_t l = strlen(inner);
      enc[a] = (char *)malloc(l + 3);
      enc[a][0] = '1';
      memcpy(enc[a] + 1, inner, l);
      enc[a][l + 1] = '0';
      enc[a][l + 2] = 0;
      free(inner);
    }
  {
    char *bits = encode_children(-1, no, par, enc);
    int nbits = (int)strlen(bits);
    if (nbits + 1 > 64 * code_words) { free(bits); rc = ORC_EOVERFLOW; goto out; }
    memset(code, 0, sizeof(uint64_t) * code_words);
    for (int b = 0; b < nbits; b++)
      if (bits[b] == '1') {
        int pos = nbits - 1 - b;
        code[pos >> 6] |= (uint64_t)1 << (pos & 63);
      }
    code[nbits >> 6] |= (uint64_t)1 << (nbits & 63);
    free(bits);
  }
  if (st) {
    int ncr = 0;
    for (int e = 0; e < c.ne; e++) ncr += crossed(&c, e);
    st->n_ovals = no;
    st->n_pseudolines = npseudo;
    st->max_depth = no ? maxd + 1 : 0;
    st->n_even = peven;
    st->n_odd = nodd;
    st->n_segments = ns;
    st->n_crossed = ncr;
    st->n_retries = retries;
  }
out:
  if (enc) { for (int a = 0; a < no; a++) free(enc[a]); free(enc); }
  free(par); free(depth); free(in); free(oval); free(segs); free(comps);
  cx_free(&c);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* batch over threads                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d, sw, cw;
  const int32_t *tri;
  const uint64_t *sig;
  uint64_t *codes;
  int32_t *status;
  orc_stats *stats;
  int64_t lo, hi, failed;
} job_t;

static void *run_job(void *arg) {
  job_t *j = (job_t *)arg;
  for (int64_t n = j->lo; n < j->hi; n++) {
    int rc = orc_real_scheme(j->d, j->tri, j->sig + n * j->sw, j->codes + n * j->cw, j->cw,
                             j->stats ? &j->stats[n] : NULL);
    if (rc) {
      j->failed++;
      memset(j->codes + n * j->cw, 0, sizeof(uint64_t) * j->cw);
    }
    if (j->status) j->status[n] = rc;
  }
  return NULL;
}

int64_t orc_real_schemes_batch(int d, const int32_t *tri, int sign_words,
                               const uint64_t *sigmas, int64_t n,
                               uint64_t *codes, int code_words,
                               int32_t *status, orc_stats *stats,
                               int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  job_t jobs[256];
  int64_t per = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; t++) {
    jobs[t] = (job_t){d, sign_words, code_words, tri, sigmas, codes, status, stats,
                      t * per, (t + 1) * per < n ? (t + 1) * per : n, 0};
    if (jobs[t].lo > n) jobs[t].lo = n;
    pthread_create(&th[t], NULL, run_job, &jobs[t]);
  }
  int64_t failed = 0;
  for (int t = 0; t < n_threads; t++) {
    pthread_join(th[t], NULL);
    failed += jobs[t].failed;
  }
  return failed;
}
