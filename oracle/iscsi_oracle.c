/*
 * iscsi_oracle.c -- plain, slow CPU oracle for the ISCI sigma-vector step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (paper_1609_07757_gb300) never calls it and shares no code,
 * header, table or helper with it.
 *
 * What it computes (Sorensen, Bauch & Madsen, arXiv:1609.07757):
 *   - the Hamiltonian in its index-restricted, spin-ordered form (Eq. index_re)
 *     H = sum_pq h_pq (a+_pa a_qa + a+_pb a_qb)
 *       + sum_{p>r,q>s} (g_psrq - g_pqrs)(a+_pa a+_ra a_qa a_sa + same for beta)
 *       - sum_pqrs g_pqrs a+_pa a+_rb a_qa a_sb
 *     with g_pqrs = (pq|rs) in chemist notation;
 *   - integral screening (Eq. sigma_int / sigma_split and the screened loops
 *     of Sec. "Second part"): a term is kept iff |unit| > tau, where the unit
 *     is h_pq, the antisymmetrised same-spin value g_psrq - g_pqrs, or the
 *     opposite-spin g_pqrs (Eq. int_share screens the antisymmetrised value);
 *   - the CI space of Eq. ci_hierarchy truncated at total excitation level k
 *     relative to the reference with the lowest orbitals occupied;
 *   - sigma = H_tau c (Eq. sigma), by two independent traversals:
 *       ora_sigma_terms : every surviving term applied to every determinant
 *                         (the distributive form of Eq. sigma_int), and
 *       ora_sigma_rows  : row-wise, H_IJ assembled from the terms that can
 *                         connect J to I (Slater-Condon selection), any n;
 *   - the one- and two-body density matrices of Eqs. d1 and d2 (Sec.
 *     "Density matrices"), spin-resolved, by explicit operator application
 *     (ora_density for all elements, ora_density_elems for single ones).
 *
 * Conventions (fixed by this library's interface, not by the paper):
 *   - strings are sorted by (excitation level, colex rank of the ascending
 *     orbital list); determinant index = off[A] + B where B runs over the
 *     beta strings with level <= k - level(A) (a prefix of the sorted list);
 *   - |A,B> = prod_{p in A ascending} a+_pa  prod_{q in B ascending} a+_qb |vac>;
 *     alpha spin-orbital p has id p, beta spin-orbital p has id n + p, so a
 *     determinant is an ascending list of spin-orbital ids, and an operator
 *     acting on id i picks up (-1)^(number of occupied ids below i).
 *   - eri is pair-packed: (pq|rs) = eri[P(p,q) * npair + P(r,s)],
 *     P(p,q) = max(p,q)(max(p,q)+1)/2 + min(p,q), npair = n(n+1)/2.
 *
 * Class ids (0..41) follow the 42 terms of Eqs. class_to_ex_dx .. the_end:
 *   0..3   one-body alpha  H^{1,1},H^{1,0},H^{0,1},H^{0,0}_{1,0,1}
 *   4..7   one-body beta   same order, H_{1,0,-1}
 *   8..23  opposite-spin terms of H_{2,0,0} (16 ex/dx combinations)
 *   24..32 alpha-alpha H^{P,H}_{2,0,2}, (P,H) = (2,2),(2,1),(1,2),(2,0),(1,1),
 *          (0,2),(1,0),(0,1),(0,0)
 *   33..41 beta-beta   H^{P,H}_{2,0,-2}, same order
 * where an orbital below n_sigma is occupied (O) and the rest virtual (V);
 * a creator in V / annihilator in O is an excitation ("ex") operator and a
 * creator in O / annihilator in V is a de-excitation ("dx") operator (Sec.
 * Theory); P counts dx annihilators and H counts dx creators.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAXE 16 /* electrons per spin */

typedef struct {
  int n, ne, count, maxlevel;
  int *orbs;          /* [count][ne], ascending, in sorted (level, colex) order */
  int *level;         /* [count] */
  int64_t *pos;       /* colex rank -> position in sorted order */
  int64_t cnt_le[ORA_MAXE + 2]; /* number of strings with level <= l */
} StrSet;

typedef struct {
  int n, na, nb, kmax;
  double tau;
  double *h1;  /* n*n */
  double *eri; /* npair*npair */
  int64_t npair;
  StrSet s[2];
  int64_t *off; /* [NA+1] */
  int64_t ndet;
} Oracle;

/* ------------------------------------------------------------------ */
/* combinatorics                                                        */

static int64_t binom64(int n, int k) {
  if (k < 0 || k > n) return 0;
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

static int64_t colex_rank(const int *o, int ne) {
  int64_t r = 0;
  for (int i = 0; i < ne; ++i) r += binom64(o[i], i + 1);
  return r;
}

static int level_of(const int *o, int ne) {
  int l = 0;
  for (int i = 0; i < ne; ++i) l += (o[i] >= ne);
  return l;
}

typedef struct {
  int level;
  int64_t colex;
  int64_t idx;
} SortKey;

static int cmp_key(const void *a, const void *b) {
  const SortKey *x = (const SortKey *)a, *y = (const SortKey *)b;
  if (x->level != y->level) return x->level < y->level ? -1 : 1;
  if (x->colex != y->colex) return x->colex < y->colex ? -1 : 1;
  return 0;
}

/* all ne-subsets of {0..n-1}, sorted by (level, colex rank) */
static int build_strings(StrSet *S, int n, int ne) {
  memset(S, 0, sizeof(*S));
  S->n = n;
  S->ne = ne;
  int64_t cnt = binom64(n, ne);
  if (cnt <= 0 || cnt > (int64_t)1 << 30) return -1;
  S->count = (int)cnt;
  int *tmp = (int *)malloc(sizeof(int) * (size_t)cnt * (ne > 0 ? ne : 1));
  SortKey *keys = (SortKey *)malloc(sizeof(SortKey) * (size_t)cnt);
  S->orbs = (int *)malloc(sizeof(int) * (size_t)cnt * (ne > 0 ? ne : 1));
  S->level = (int *)malloc(sizeof(int) * (size_t)cnt);
  S->pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt);
  if (!tmp || !keys || !S->orbs || !S->level || !S->pos) return -2;
  int c[ORA_MAXE];
  for (int i = 0; i < ne; ++i) c[i] = i;
  for (int64_t k = 0; k < cnt; ++k) {
    memcpy(tmp + k * ne, c, sizeof(int) * ne);
    keys[k].level = level_of(c, ne);
    keys[k].colex = colex_rank(c, ne);
    keys[k].idx = k;
    /* next combination in lexicographic order */
    int i = ne - 1;
    while (i >= 0 && c[i] == n - ne + i) --i;
    if (i < 0) break;
    ++c[i];
    for (int j = i + 1; j < ne; ++j) c[j] = c[j - 1] + 1;
  }
  qsort(keys, (size_t)cnt, sizeof(SortKey), cmp_key);
  S->maxlevel = 0;
  for (int64_t k = 0; k < cnt; ++k) {
    memcpy(S->orbs + k * ne, tmp + keys[k].idx * ne, sizeof(int) * ne);
    S->level[k] = keys[k].level;
    S->pos[keys[k].colex] = k;
    if (keys[k].level > S->maxlevel) S->maxlevel = keys[k].level;
  }
  for (int l = 0; l < ORA_MAXE + 2; ++l) S->cnt_le[l] = 0;
  for (int64_t k = 0; k < cnt; ++k)
    for (int l = S->level[k]; l < ORA_MAXE + 2; ++l) S->cnt_le[l]++;
  free(tmp);
  free(keys);
  return 0;
}

static void free_strings(StrSet *S) {
  free(S->orbs);
  free(S->level);
  free(S->pos);
}

/* number of beta strings allowed beside an alpha string of level la */
static int64_t nb_allowed(const Oracle *o, int la) {
  int rem = o->kmax - la;
  if (rem < 0) return 0;
  if (rem > ORA_MAXE + 1) rem = ORA_MAXE + 1;
  return o->s[1].cnt_le[rem];
}

/* ------------------------------------------------------------------ */
/* second-quantised operators acting on an ascending spin-orbital list  */

typedef struct {
  int len;
  int so[2 * ORA_MAXE];
} Det;

/* returns +1/-1, or 0 if the result vanishes */
static int op_apply(Det *d, int create, int so) {
  int pos = 0;
  while (pos < d->len && d->so[pos] < so) ++pos;
  int present = (pos < d->len && d->so[pos] == so);
  if (create) {
    if (present) return 0;
    for (int j = d->len; j > pos; --j) d->so[j] = d->so[j - 1];
    d->so[pos] = so;
    d->len++;
  } else {
    if (!present) return 0;
    for (int j = pos; j < d->len - 1; ++j) d->so[j] = d->so[j + 1];
    d->len--;
  }
  return (pos & 1) ? -1 : 1;
}

typedef struct {
  int nops;
  int create[4];
  int so[4];
} OpString; /* operators written left to right; applied right to left */

static int opstring_apply(const OpString *op, Det *d) {
  int sign = 1;
  for (int i = op->nops - 1; i >= 0; --i) {
    int s = op_apply(d, op->create[i], op->so[i]);
    if (!s) return 0;
    sign *= s;
  }
  return sign;
}

static void det_from(const Oracle *o, int64_t ia, int64_t ib, Det *d) {
  const StrSet *A = &o->s[0], *B = &o->s[1];
  d->len = 0;
  for (int i = 0; i < A->ne; ++i) d->so[d->len++] = A->orbs[ia * A->ne + i];
  for (int i = 0; i < B->ne; ++i) d->so[d->len++] = o->n + B->orbs[ib * B->ne + i];
}

/* index of a determinant given as an ascending spin-orbital list, or -1 */
static int64_t det_lookup(const Oracle *o, const Det *d) {
  int a[ORA_MAXE], b[ORA_MAXE], na = 0, nb = 0;
  for (int i = 0; i < d->len; ++i) {
    if (d->so[i] < o->n) {
      if (na >= ORA_MAXE) return -1;
      a[na++] = d->so[i];
    } else {
      if (nb >= ORA_MAXE) return -1;
      b[nb++] = d->so[i] - o->n;
    }
  }
  if (na != o->na || nb != o->nb) return -1;
  int64_t ia = o->s[0].pos[colex_rank(a, na)];
  int64_t ib = o->s[1].pos[colex_rank(b, nb)];
  if (ib >= nb_allowed(o, o->s[0].level[ia])) return -1;
  return o->off[ia] + ib;
}

/* ------------------------------------------------------------------ */
/* integrals, units and classes                                         */

static double g_at(const Oracle *o, int p, int q, int r, int s) {
  if (!o->eri) return 0.0;
  int64_t pq = p >= q ? (int64_t)p * (p + 1) / 2 + q : (int64_t)q * (q + 1) / 2 + p;
  int64_t rs = r >= s ? (int64_t)r * (r + 1) / 2 + s : (int64_t)s * (s + 1) / 2 + r;
  return o->eri[pq * o->npair + rs];
}

/* spin-part kind: 0 = C^dx A^ex (OO), 1 = C^dx A^dx, 2 = C^ex A^ex, 3 = C^ex A^dx (VV) */
static int kind_of(int creator_virtual, int annihilator_virtual) {
  return 2 * creator_virtual + annihilator_virtual;
}

static int class_onebody(int spin, int pv, int qv) {
  static const int order[4] = {2, 0, 3, 1}; /* kind -> position in H^{1,1},H^{1,0},H^{0,1},H^{0,0} */
  return 4 * spin + order[kind_of(pv, qv)];
}

static int class_opposite(int pv, int qv, int rv, int sv) {
  /* (alpha kind, beta kind) of the 16 opposite-spin terms, listed in the
     order H^{2,2}, H^{2,1} a,b, H^{1,2} a,b, H^{2,0}, H^{1,1} a..d, H^{0,2},
     H^{1,0} a,b, H^{0,1} a,b, H^{0,0} */
  static const int ka[16] = {1, 3, 1, 0, 1, 3, 1, 0, 3, 2, 0, 2, 3, 2, 0, 2};
  static const int kb[16] = {1, 1, 3, 1, 0, 3, 2, 3, 0, 1, 0, 3, 2, 0, 2, 2};
  int a = kind_of(pv, qv), b = kind_of(rv, sv);
  for (int t = 0; t < 16; ++t)
    if (ka[t] == a && kb[t] == b) return 8 + t;
  return -1;
}

static int class_samespin(int spin, int pv, int rv, int qv, int sv) {
  static const int P_of[9] = {2, 2, 1, 2, 1, 0, 1, 0, 0};
  static const int H_of[9] = {2, 1, 2, 0, 1, 2, 0, 1, 0};
  int P = qv + sv;             /* annihilators in V are dx */
  int H = (!pv) + (!rv);       /* creators in O are dx */
  for (int t = 0; t < 9; ++t)
    if (P_of[t] == P && H_of[t] == H) return 24 + 9 * spin + t;
  return -1;
}

static int in_mask(uint64_t mask, int cls) { return cls >= 0 && ((mask >> cls) & 1ull); }

static int keep(const Oracle *o, double u) { return fabs(u) > o->tau; }

/* ------------------------------------------------------------------ */
/* public: construction                                                 */

void *ora_create(int n, int na, int nb, int kmax, double tau, const double *h1, const double *eri) {
  if (n <= 0 || na < 0 || nb < 0 || na > n || nb > n || na > ORA_MAXE || nb > ORA_MAXE || tau < 0) return NULL;
  Oracle *o = (Oracle *)calloc(1, sizeof(Oracle));
  o->n = n;
  o->na = na;
  o->nb = nb;
  o->kmax = kmax;
  o->tau = tau;
  o->npair = (int64_t)n * (n + 1) / 2;
  o->h1 = (double *)malloc(sizeof(double) * n * n);
  memcpy(o->h1, h1, sizeof(double) * n * n);
  if (eri) {
    o->eri = (double *)malloc(sizeof(double) * (size_t)(o->npair * o->npair));
    memcpy(o->eri, eri, sizeof(double) * (size_t)(o->npair * o->npair));
  } else {
    o->eri = NULL; /* no two-electron part */
  }
  if (build_strings(&o->s[0], n, na) || build_strings(&o->s[1], n, nb)) return NULL;
  o->off = (int64_t *)malloc(sizeof(int64_t) * (o->s[0].count + 1));
  o->off[0] = 0;
  for (int a = 0; a < o->s[0].count; ++a) o->off[a + 1] = o->off[a] + nb_allowed(o, o->s[0].level[a]);
  o->ndet = o->off[o->s[0].count];
  return o;
}

void ora_destroy(void *p) {
  Oracle *o = (Oracle *)p;
  if (!o) return;
  free_strings(&o->s[0]);
  free_strings(&o->s[1]);
  free(o->off);
  free(o->h1);
  free(o->eri);
  free(o);
}

int64_t ora_ndet(void *p) { return ((Oracle *)p)->ndet; }

int ora_nstrings(void *p, int spin) { return ((Oracle *)p)->s[spin].count; }

void ora_strings(void *p, int spin, int *orbs, int *levels) {
  Oracle *o = (Oracle *)p;
  StrSet *S = &o->s[spin];
  memcpy(orbs, S->orbs, sizeof(int) * (size_t)S->count * S->ne);
  memcpy(levels, S->level, sizeof(int) * (size_t)S->count);
}

void ora_offsets(void *p, int64_t *off) {
  Oracle *o = (Oracle *)p;
  memcpy(off, o->off, sizeof(int64_t) * (o->s[0].count + 1));
}

/* determinant index from ascending alpha / beta orbital lists, -1 if outside */
int64_t ora_det_index(void *p, const int *aorbs, const int *borbs) {
  Oracle *o = (Oracle *)p;
  Det d;
  d.len = 0;
  for (int i = 0; i < o->na; ++i) d.so[d.len++] = aorbs[i];
  for (int i = 0; i < o->nb; ++i) d.so[d.len++] = o->n + borbs[i];
  return det_lookup(o, &d);
}

/* (alpha string position, beta string position) of a determinant index */
static void det_split(const Oracle *o, int64_t I, int64_t *ia, int64_t *ib) {
  int64_t lo = 0, hi = o->s[0].count - 1;
  while (lo < hi) { /* last a with off[a] <= I */
    int64_t mid = (lo + hi + 1) / 2;
    if (o->off[mid] <= I) lo = mid;
    else hi = mid - 1;
  }
  while (o->off[lo + 1] == o->off[lo]) ++lo; /* skip alpha strings with no beta allowed */
  *ia = lo;
  *ib = I - o->off[lo];
}

/* ------------------------------------------------------------------ */
/* sigma by applying every surviving term to every determinant          */

typedef struct {
  const Oracle *o;
  const double *c;
  double *sigma;
  int64_t updates;
} TermCtx;

static void apply_term_all(TermCtx *t, const OpString *op, double coef) {
  const Oracle *o = t->o;
  for (int64_t ia = 0; ia < o->s[0].count; ++ia) {
    int64_t nbj = nb_allowed(o, o->s[0].level[ia]);
    for (int64_t ib = 0; ib < nbj; ++ib) {
      int64_t J = o->off[ia] + ib;
      Det d;
      det_from(o, ia, ib, &d);
      int sg = opstring_apply(op, &d);
      if (!sg) continue;
      int64_t I = det_lookup(o, &d);
      if (I < 0) continue;
      t->sigma[I] += coef * sg * t->c[J];
      t->updates++;
    }
  }
}

void ora_sigma_terms(void *p, const double *c, double *sigma, uint64_t mask, int64_t *nupdates) {
  Oracle *o = (Oracle *)p;
  int n = o->n;
  TermCtx t = {o, c, sigma, 0};
  for (int64_t I = 0; I < o->ndet; ++I) sigma[I] = 0.0;
  int nel[2] = {o->na, o->nb};
  /* one-body: h_pq (a+_p a_q) for each spin */
  for (int spin = 0; spin < 2; ++spin) {
    int ne = nel[spin];
    for (int pp = 0; pp < n; ++pp)
      for (int q = 0; q < n; ++q) {
        double u = o->h1[pp * n + q];
        if (!keep(o, u) || !in_mask(mask, class_onebody(spin, pp >= ne, q >= ne))) continue;
        OpString op = {2, {1, 0, 0, 0}, {spin * n + pp, spin * n + q, 0, 0}};
        apply_term_all(&t, &op, u);
      }
  }
  /* same-spin: (g_psrq - g_pqrs) a+_p a+_r a_q a_s, p>r, q>s */
  for (int spin = 0; spin < 2; ++spin) {
    int ne = nel[spin];
    for (int pp = 0; pp < n; ++pp)
      for (int r = 0; r < pp; ++r)
        for (int q = 0; q < n; ++q)
          for (int s = 0; s < q; ++s) {
            double u = g_at(o, pp, s, r, q) - g_at(o, pp, q, r, s);
            if (!keep(o, u) || !in_mask(mask, class_samespin(spin, pp >= ne, r >= ne, q >= ne, s >= ne))) continue;
            OpString op = {4, {1, 1, 0, 0}, {spin * n + pp, spin * n + r, spin * n + q, spin * n + s}};
            apply_term_all(&t, &op, u);
          }
  }
  /* opposite-spin: -g_pqrs a+_pa a+_rb a_qa a_sb */
  for (int pp = 0; pp < n; ++pp)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
          double u = g_at(o, pp, q, r, s);
          if (!keep(o, u) || !in_mask(mask, class_opposite(pp >= o->na, q >= o->na, r >= o->nb, s >= o->nb))) continue;
          OpString op = {4, {1, 1, 0, 0}, {pp, n + r, q, n + s}};
          apply_term_all(&t, &op, -u);
        }
  if (nupdates) *nupdates = t.updates;
}

/* ------------------------------------------------------------------ */
/* H_IJ from the terms that can connect J to I (Slater-Condon selection) */

static int det_equal(const Det *a, const Det *b) {
  if (a->len != b->len) return 0;
  for (int i = 0; i < a->len; ++i)
    if (a->so[i] != b->so[i]) return 0;
  return 1;
}

/* contribution of one term to <I| term |J>; 0 if screened or not connecting */
static double term_elem(const Oracle *o, const Det *dI, const Det *dJ, const OpString *op, double coef, double u,
                        int cls, uint64_t mask) {
  if (!keep(o, u) || !in_mask(mask, cls)) return 0.0;
  Det d = *dJ;
  int sg = opstring_apply(op, &d);
  if (!sg || !det_equal(&d, dI)) return 0.0;
  return coef * sg * u;
}

static void split_spin(const Oracle *o, const Det *d, int *a, int *b) {
  int na = 0, nb = 0;
  for (int i = 0; i < d->len; ++i) {
    if (d->so[i] < o->n) a[na++] = d->so[i];
    else b[nb++] = d->so[i] - o->n;
  }
}

static int contains(const int *x, int len, int v) {
  for (int i = 0; i < len; ++i)
    if (x[i] == v) return 1;
  return 0;
}

/* elements of x not in y */
static int set_minus(const int *x, int lx, const int *y, int ly, int *out) {
  int k = 0;
  for (int i = 0; i < lx; ++i)
    if (!contains(y, ly, x[i])) out[k++] = x[i];
  return k;
}

static double samespin_term(const Oracle *o, const Det *dI, const Det *dJ, int spin, int c1, int c2, int a1, int a2,
                            uint64_t mask) {
  /* creators {c1,c2} ordered p>r, annihilators {a1,a2} ordered q>s */
  int n = o->n, ne = spin ? o->nb : o->na;
  int pp = c1 > c2 ? c1 : c2, r = c1 > c2 ? c2 : c1;
  int q = a1 > a2 ? a1 : a2, s = a1 > a2 ? a2 : a1;
  if (pp == r || q == s) return 0.0;
  double u = g_at(o, pp, s, r, q) - g_at(o, pp, q, r, s);
  OpString op = {4, {1, 1, 0, 0}, {spin * n + pp, spin * n + r, spin * n + q, spin * n + s}};
  return term_elem(o, dI, dJ, &op, 1.0, u, class_samespin(spin, pp >= ne, r >= ne, q >= ne, s >= ne), mask);
}

static double onebody_term(const Oracle *o, const Det *dI, const Det *dJ, int spin, int pp, int q, uint64_t mask) {
  int n = o->n, ne = spin ? o->nb : o->na;
  OpString op = {2, {1, 0, 0, 0}, {spin * n + pp, spin * n + q, 0, 0}};
  return term_elem(o, dI, dJ, &op, 1.0, o->h1[pp * n + q], class_onebody(spin, pp >= ne, q >= ne), mask);
}

static double opposite_term(const Oracle *o, const Det *dI, const Det *dJ, int pp, int q, int r, int s, uint64_t mask) {
  int n = o->n;
  OpString op = {4, {1, 1, 0, 0}, {pp, n + r, q, n + s}};
  return term_elem(o, dI, dJ, &op, -1.0, g_at(o, pp, q, r, s),
                   class_opposite(pp >= o->na, q >= o->na, r >= o->nb, s >= o->nb), mask);
}

static double hij(const Oracle *o, const Det *dI, const Det *dJ, uint64_t mask) {
  int aI[ORA_MAXE], bI[ORA_MAXE], aJ[ORA_MAXE], bJ[ORA_MAXE];
  split_spin(o, dI, aI, bI);
  split_spin(o, dJ, aJ, bJ);
  int na = o->na, nb = o->nb;
  int pa[ORA_MAXE], qa[ORA_MAXE], pb[ORA_MAXE], qb[ORA_MAXE];
  int da = set_minus(aI, na, aJ, na, pa); /* created alpha (in I, not J) */
  set_minus(aJ, na, aI, na, qa);          /* annihilated alpha */
  int db = set_minus(bI, nb, bJ, nb, pb);
  set_minus(bJ, nb, bI, nb, qb);
  double h = 0.0;
  if (da + db > 2) return 0.0;
  if (da == 0 && db == 0) {
    for (int i = 0; i < na; ++i) h += onebody_term(o, dI, dJ, 0, aI[i], aI[i], mask);
    for (int i = 0; i < nb; ++i) h += onebody_term(o, dI, dJ, 1, bI[i], bI[i], mask);
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < i; ++j) h += samespin_term(o, dI, dJ, 0, aI[i], aI[j], aI[i], aI[j], mask);
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < i; ++j) h += samespin_term(o, dI, dJ, 1, bI[i], bI[j], bI[i], bI[j], mask);
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < nb; ++j) h += opposite_term(o, dI, dJ, aI[i], aI[i], bI[j], bI[j], mask);
  } else if (da == 1 && db == 0) {
    int pp = pa[0], q = qa[0];
    h += onebody_term(o, dI, dJ, 0, pp, q, mask);
    for (int i = 0; i < na; ++i) {
      int k = aJ[i];
      if (k == q) continue;
      h += samespin_term(o, dI, dJ, 0, pp, k, q, k, mask);
    }
    for (int j = 0; j < nb; ++j) h += opposite_term(o, dI, dJ, pp, q, bJ[j], bJ[j], mask);
  } else if (da == 0 && db == 1) {
    int pp = pb[0], q = qb[0];
    h += onebody_term(o, dI, dJ, 1, pp, q, mask);
    for (int i = 0; i < nb; ++i) {
      int k = bJ[i];
      if (k == q) continue;
      h += samespin_term(o, dI, dJ, 1, pp, k, q, k, mask);
    }
    for (int j = 0; j < na; ++j) h += opposite_term(o, dI, dJ, aJ[j], aJ[j], pp, q, mask);
  } else if (da == 2) {
    h += samespin_term(o, dI, dJ, 0, pa[0], pa[1], qa[0], qa[1], mask);
  } else if (db == 2) {
    h += samespin_term(o, dI, dJ, 1, pb[0], pb[1], qb[0], qb[1], mask);
  } else { /* da == 1 && db == 1 */
    h += opposite_term(o, dI, dJ, pa[0], qa[0], pb[0], qb[0], mask);
  }
  return h;
}

static void det_of_index(const Oracle *o, int64_t I, Det *d) {
  int64_t ia, ib;
  det_split(o, I, &ia, &ib);
  det_from(o, ia, ib, d);
}

/* one matrix element H_IJ */
double ora_hij(void *p, int64_t I, int64_t J, uint64_t mask) {
  Oracle *o = (Oracle *)p;
  Det dI, dJ;
  det_of_index(o, I, &dI);
  det_of_index(o, J, &dJ);
  return hij(o, &dI, &dJ, mask);
}

/* dense H (ndet x ndet, row-major); small spaces only */
void ora_dense_h(void *p, double *H, uint64_t mask) {
  Oracle *o = (Oracle *)p;
  int64_t N = o->ndet;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t I = 0; I < N; ++I) {
    Det dI, dJ;
    det_of_index(o, I, &dI);
    for (int64_t J = 0; J < N; ++J) {
      det_of_index(o, J, &dJ);
      H[I * N + J] = hij(o, &dI, &dJ, mask);
    }
  }
}

/* callback over all determinants J connected to I by <= 2 replacements */
typedef struct {
  const Oracle *o;
  const double *c;
  uint64_t mask;
  const Det *dI;
  double acc;
} RowCtx;

static void row_visit(RowCtx *rc, const Det *dJ) {
  int64_t J = det_lookup(rc->o, dJ);
  if (J < 0) return;
  double h = hij(rc->o, rc->dI, dJ, rc->mask);
  if (h != 0.0) rc->acc += h * rc->c[J];
}

/* replace orbital at index i of spin list by v (keeps list ascending) */
static void make_det(const Oracle *o, const int *a, const int *b, Det *d) {
  int ta[ORA_MAXE], tb[ORA_MAXE];
  memcpy(ta, a, sizeof(int) * o->na);
  memcpy(tb, b, sizeof(int) * o->nb);
  /* insertion sort */
  for (int i = 1; i < o->na; ++i)
    for (int j = i; j > 0 && ta[j - 1] > ta[j]; --j) {
      int t = ta[j];
      ta[j] = ta[j - 1];
      ta[j - 1] = t;
    }
  for (int i = 1; i < o->nb; ++i)
    for (int j = i; j > 0 && tb[j - 1] > tb[j]; --j) {
      int t = tb[j];
      tb[j] = tb[j - 1];
      tb[j - 1] = t;
    }
  d->len = 0;
  for (int i = 0; i < o->na; ++i) d->so[d->len++] = ta[i];
  for (int i = 0; i < o->nb; ++i) d->so[d->len++] = o->n + tb[i];
}

static double sigma_row(const Oracle *o, const double *c, int64_t I, uint64_t mask) {
  int n = o->n, na = o->na, nb = o->nb;
  Det dI, dJ;
  det_of_index(o, I, &dI);
  int a[ORA_MAXE], b[ORA_MAXE], ta[ORA_MAXE], tb[ORA_MAXE];
  split_spin(o, &dI, a, b);
  RowCtx rc = {o, c, mask, &dI, 0.0};
  row_visit(&rc, &dI); /* diagonal */
  /* alpha singles */
  for (int i = 0; i < na; ++i)
    for (int v = 0; v < n; ++v) {
      if (contains(a, na, v)) continue;
      memcpy(ta, a, sizeof(int) * na);
      ta[i] = v;
      make_det(o, ta, b, &dJ);
      row_visit(&rc, &dJ);
    }
  /* beta singles */
  for (int i = 0; i < nb; ++i)
    for (int v = 0; v < n; ++v) {
      if (contains(b, nb, v)) continue;
      memcpy(tb, b, sizeof(int) * nb);
      tb[i] = v;
      make_det(o, a, tb, &dJ);
      row_visit(&rc, &dJ);
    }
  /* alpha-alpha doubles */
  for (int i = 0; i < na; ++i)
    for (int j = i + 1; j < na; ++j)
      for (int v = 0; v < n; ++v) {
        if (contains(a, na, v)) continue;
        for (int w = v + 1; w < n; ++w) {
          if (contains(a, na, w)) continue;
          memcpy(ta, a, sizeof(int) * na);
          ta[i] = v;
          ta[j] = w;
          make_det(o, ta, b, &dJ);
          row_visit(&rc, &dJ);
        }
      }
  /* beta-beta doubles */
  for (int i = 0; i < nb; ++i)
    for (int j = i + 1; j < nb; ++j)
      for (int v = 0; v < n; ++v) {
        if (contains(b, nb, v)) continue;
        for (int w = v + 1; w < n; ++w) {
          if (contains(b, nb, w)) continue;
          memcpy(tb, b, sizeof(int) * nb);
          tb[i] = v;
          tb[j] = w;
          make_det(o, a, tb, &dJ);
          row_visit(&rc, &dJ);
        }
      }
  /* alpha-beta doubles */
  for (int i = 0; i < na; ++i)
    for (int v = 0; v < n; ++v) {
      if (contains(a, na, v)) continue;
      memcpy(ta, a, sizeof(int) * na);
      ta[i] = v;
      for (int j = 0; j < nb; ++j)
        for (int w = 0; w < n; ++w) {
          if (contains(b, nb, w)) continue;
          memcpy(tb, b, sizeof(int) * nb);
          tb[j] = w;
          make_det(o, ta, tb, &dJ);
          row_visit(&rc, &dJ);
        }
    }
  return rc.acc;
}

/* sigma_I for the listed rows (any size); nthreads <= 0 uses the default */
void ora_sigma_rows(void *p, const double *c, const int64_t *rows, int64_t nrows, double *out, uint64_t mask,
                    int nthreads) {
  Oracle *o = (Oracle *)p;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t k = 0; k < nrows; ++k) out[k] = sigma_row(o, c, rows[k], mask);
}

/* ------------------------------------------------------------------ */
/* density matrices (Sec. "Density matrices", Eqs. d1 and d2)           */
/*                                                                      */
/* Spin-resolved blocks, from the definitions by explicit operator      */
/* application on every determinant of the space (no string tables, no  */
/* excitation classes):                                                 */
/*   D1[s][p][q]     = <bra| a+_{p s} a_{q s} |ket>,     s = alpha, beta   */
/*   D2[b][p][q][r][t] = <bra| a+_{p s} a+_{r u} a_{t u} a_{q s} |ket>     */
/*     with (s, u) = (alpha, alpha), (alpha, beta), (beta, beta) for       */
/*     b = 0, 1, 2; flat index ((p n + q) n + r) n + t.                   */
/* The spin-summed D2 of Eq. d2 is D2[0] + D2[2] + D2[1] + D2[1] with     */
/* (p,q) and (r,t) swapped.                                             */

static const int dm_spin1[3] = {0, 0, 1}, dm_spin2[3] = {0, 1, 1};

/* accumulates ket_J's contributions into d1 [2 n n] and d2 [3 n^4] (d2 may be NULL) */
static void density_from_det(const Oracle *o, const double *bra, double kJ, const Det *dJ, double *d1, double *d2) {
  int n = o->n;
  for (int sp = 0; sp < 2; ++sp)
    for (int q = 0; q < n; ++q) {
      Det d0 = *dJ;
      int s1 = op_apply(&d0, 0, sp * n + q);
      if (!s1) continue;
      for (int p = 0; p < n; ++p) {
        Det d = d0;
        int s2 = op_apply(&d, 1, sp * n + p);
        if (!s2) continue;
        int64_t I = det_lookup(o, &d);
        if (I >= 0) d1[(sp * n + p) * n + q] += bra[I] * (double)(s1 * s2) * kJ;
      }
    }
  if (!d2) return;
  int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
  for (int b = 0; b < 3; ++b) {
    int so1 = dm_spin1[b] * n, so2 = dm_spin2[b] * n;
    for (int q = 0; q < n; ++q)
      for (int t = 0; t < n; ++t) {
        Det d0 = *dJ; /* a_{q s} acts first, then a_{t u} */
        int s1 = op_apply(&d0, 0, so1 + q);
        if (!s1) continue;
        int s2 = op_apply(&d0, 0, so2 + t);
        if (!s2) continue;
        for (int r = 0; r < n; ++r) {
          Det d1r = d0;
          int s3 = op_apply(&d1r, 1, so2 + r);
          if (!s3) continue;
          for (int p = 0; p < n; ++p) {
            Det d = d1r;
            int s4 = op_apply(&d, 1, so1 + p);
            if (!s4) continue;
            int64_t I = det_lookup(o, &d);
            if (I < 0) continue;
            d2[b * n4 + ((int64_t)p * n + q) * n2 + (int64_t)r * n + t] += bra[I] * (double)(s1 * s2 * s3 * s4) * kJ;
          }
        }
      }
  }
}

/* all blocks of D1 and (if d2) D2 for the pair (bra, ket); both [ndet] */
void ora_density(void *ptr, const double *bra, const double *ket, double *d1, double *d2, int nthreads) {
  Oracle *o = (Oracle *)ptr;
  int n = o->n;
  int64_t n1 = 2 * (int64_t)n * n, n4 = (int64_t)n * n * n * n, n2tot = d2 ? 3 * n4 : 0;
  memset(d1, 0, sizeof(double) * (size_t)n1);
  if (d2) memset(d2, 0, sizeof(double) * (size_t)n2tot);
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
  /* private accumulators: at most ~2 GB in total */
  int64_t per = (n1 + n2tot) * (int64_t)sizeof(double);
  while (nt > 1 && per * nt > ((int64_t)2 << 30)) --nt;
#else
  (void)nthreads;
#endif
  double *acc = (double *)calloc((size_t)nt * (size_t)(n1 + n2tot), sizeof(double));
  if (!acc) return;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
#endif
  for (int64_t J = 0; J < o->ndet; ++J) {
    if (ket[J] == 0.0) continue;
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *a1 = acc + (size_t)tid * (size_t)(n1 + n2tot);
    Det dJ;
    det_of_index(o, J, &dJ);
    density_from_det(o, bra, ket[J], &dJ, a1, d2 ? a1 + n1 : NULL);
  }
  for (int t = 0; t < nt; ++t) {
    double *a1 = acc + (size_t)t * (size_t)(n1 + n2tot);
    for (int64_t i = 0; i < n1; ++i) d1[i] += a1[i];
    for (int64_t i = 0; i < n2tot; ++i) d2[i] += a1[n1 + i];
  }
  free(acc);
}

/* single elements, each summed over every determinant J of the space:
   spec[5k..5k+4] = (block, p, q, r, t); block 0..2 are the D2 blocks
   (aa, ab, bb), block 3 / 4 the alpha / beta D1 (r, t ignored) */
void ora_density_elems(void *ptr, const double *bra, const double *ket, const int *spec, int64_t m, double *out,
                       int nthreads) {
  Oracle *o = (Oracle *)ptr;
  int n = o->n;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < m; ++k) {
    const int *sp = spec + 5 * k;
    OpString op;
    if (sp[0] >= 3) {
      int s = (sp[0] - 3) * n;
      op.nops = 2;
      op.create[0] = 1;
      op.so[0] = s + sp[1];
      op.create[1] = 0;
      op.so[1] = s + sp[2];
    } else {
      int s1 = dm_spin1[sp[0]] * n, s2 = dm_spin2[sp[0]] * n;
      op.nops = 4;
      op.create[0] = 1;
      op.so[0] = s1 + sp[1];
      op.create[1] = 1;
      op.so[1] = s2 + sp[3];
      op.create[2] = 0;
      op.so[2] = s2 + sp[4];
      op.create[3] = 0;
      op.so[3] = s1 + sp[2];
    }
    double acc = 0.0;
    for (int64_t J = 0; J < o->ndet; ++J) {
      if (ket[J] == 0.0) continue;
      Det d;
      det_of_index(o, J, &d);
      int sg = opstring_apply(&op, &d);
      if (!sg) continue;
      int64_t I = det_lookup(o, &d);
      if (I >= 0) acc += bra[I] * (double)sg * ket[J];
    }
    out[k] = acc;
  }
}

int ora_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* apply an operator string (written left to right, applied right to left) to
   an ascending list of spin-orbital ids; returns the sign, 0 if it vanishes */
int ora_apply(int nops, const int *create, const int *so, int len, const int *in, int *out, int *outlen) {
  if (nops > 4 || len > 2 * ORA_MAXE) return 0;
  Det d;
  d.len = len;
  for (int i = 0; i < len; ++i) d.so[i] = in[i];
  OpString op;
  op.nops = nops;
  for (int i = 0; i < nops; ++i) {
    op.create[i] = create[i];
    op.so[i] = so[i];
  }
  int sg = opstring_apply(&op, &d);
  *outlen = d.len;
  for (int i = 0; i < d.len; ++i) out[i] = d.so[i];
  return sg;
}
