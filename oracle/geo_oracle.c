/*
 * geo_oracle.c -- TEST INFRASTRUCTURE. Plain, slow, scalar FP64 CPU oracle for
 * the vector navigator of "Vectorising the detector geometry to optimize
 * particle transport" (Apostolakis, Brun, Carminati, Gheata, Wenzel).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code, header, table or constant with
 * the CUDA path; it is compiled with -O2 -ffp-contract=off (no implicit FMA,
 * no fast-math) so it gives the same bits on every host.
 *
 * What it computes (Sec. 3, Fig. 1 and Sec. 3.1):
 *   - DistFromOutside / DistFromInside of Box, Tube, Cone (Sec. 3.1, Fig. 2)
 *   - Contains (inside/outside check) and Safety (Sec. 3.1)
 *   - the navigator of Fig. 1: mother DistFromInside, then for every daughter
 *     master->local transform + DistFromOutside, then min and hit index
 *     (Sec. 3, Sec. 3.1 "coordinate transformations ... min/max algorithms")
 *   - the adjoint of the navigator step (not in the paper; implicit-function
 *     rule on the winning surface).
 *
 * Method: every distance is the plain set definition written out.  For the
 * line x + s*u the oracle builds the exact set S = { s in R : x + s*u in solid }
 * as a sorted list of closed intervals (intersection of one slab and up to
 * two quadratic constraints) and reads
 *     DistFromOutside = inf (S intersect [0, inf))          (+inf if empty)
 *     DistFromInside  = sup of the component of S intersect [0, inf) holding 0
 *                       (0 if x is outside).
 * Solids are closed sets; no tolerance enters a definition.
 *
 * Readings where the paper is silent (the paper defers shapes to ROOT):
 *   Box  params (dx,dy,dz) half-lengths.
 *   Tube params (rmin,rmax,dz); solid when rmin == 0.
 *   Cone params (dz,rmin1,rmax1,rmin2,rmax2), index 1 at z=-dz, 2 at z=+dz.
 *   Tube segment (rmin,rmax,dz,sphi,dphi): the tube cut to the closed wedge
 *     of azimuths [sphi, sphi+dphi], 0 < dphi <= 2 pi (2 pi: the whole tube);
 *     the wedge is the intersection (dphi <= pi) or the union (dphi > pi) of
 *     the half-planes n1.(x,y) >= 0, n1 = (-sin sphi, cos sphi), and
 *     n2.(x,y) >= 0, n2 = (sin(sphi+dphi), -cos(sphi+dphi)); it holds the axis.
 *   Polycone (Sec. 3.1, the sequence of connected cone and tube sections):
 *     nz z-planes z[0] < ... < z[nz-1] with inner and outer radii rmin[k] <=
 *     rmax[k] at plane k; section k (between planes k and k+1) is the cone
 *     whose radii vary linearly from plane k to plane k+1, and the solid is
 *     the union of its sections cut to the wedge [sphi, sphi+dphi] (as for
 *     the tube segment).  Neighbouring sections share the annulus of their
 *     common plane, so the inner planes are no surfaces.  The shape routines
 *     read the block [sphi, dphi, nz, z[nz], rmin[nz], rmax[nz]].
 *   Placement p_mother = R p_local + t, R row-major.
 *   Miss = +inf.  Ties: mother first, then lowest daughter index.
 *   Track outside the mother: step 0, hit -2.  Zero/non-finite input: NaN, -2.
 *   Safety is the exact Euclidean distance to the nearest boundary.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define K_BOX 0
#define K_TUBE 1
#define K_CONE 2
#define K_TUBS 3   /* tube segment: (rmin, rmax, dz, sphi, dphi) */

/* Surface (face) tags carried on interval endpoints.  Box faces 0..5 are
 * -x,+x,-y,+y,-z,+z; tubes and cones use 4/5 for -z/+z, 6 outer, 7 inner. */
#define F_NONE (-1)
#define F_ZM 4
#define F_ZP 5
#define F_OUT 6
#define F_IN 7
#define F_PHI1 8   /* tube segment: the face at sphi        */
#define F_PHI2 9   /* tube segment: the face at sphi + dphi */
#define K_PCON 4   /* polycone: block (sphi, dphi, nz, z[], rmin[], rmax[]) */
#define F_SEC 16   /* polycone: outer surface of section k = 16 + 2k, inner 17 + 2k */
#define MAXZ 32    /* polycone: at most 32 planes */

typedef struct {
    double lo, hi;
    int flo, fhi;     /* surface tag of each endpoint                      */
    double clo, chi;  /* half-chord sqrt(D)/|A| of a quadratic endpoint
                         (+inf for planes): conditioning of that endpoint */
} ivl;

#define MAXI 64
typedef struct { int n; ivl v[MAXI]; } iset;

static void set_copy(iset *dst, const iset *src) {
    dst->n = src->n;
    memcpy(dst->v, src->v, (size_t)src->n * sizeof(ivl));
}

static void set_all(iset *s) {
    s->n = 1;
    s->v[0].lo = -INFINITY; s->v[0].hi = INFINITY;
    s->v[0].flo = s->v[0].fhi = F_NONE;
    s->v[0].clo = s->v[0].chi = INFINITY;
}
static void set_empty(iset *s) { s->n = 0; }

static void set_one(iset *s, double lo, int flo, double clo, double hi, int fhi, double chi) {
    s->n = 1;
    s->v[0].lo = lo; s->v[0].flo = flo; s->v[0].clo = clo;
    s->v[0].hi = hi; s->v[0].fhi = fhi; s->v[0].chi = chi;
}

/* a <- a intersect b, both sorted lists of disjoint closed intervals. */
static void set_and(iset *a, const iset *b) {
    iset r; r.n = 0;
    int i = 0, j = 0;
    while (i < a->n && j < b->n) {
        const ivl *x = &a->v[i], *y = &b->v[j];
        ivl z;
        if (x->lo >= y->lo) { z.lo = x->lo; z.flo = x->flo; z.clo = x->clo; }
        else                { z.lo = y->lo; z.flo = y->flo; z.clo = y->clo; }
        if (x->hi <= y->hi) { z.hi = x->hi; z.fhi = x->fhi; z.chi = x->chi; }
        else                { z.hi = y->hi; z.fhi = y->fhi; z.chi = y->chi; }
        if (z.lo <= z.hi) {
            if (r.n >= MAXI) abort();
            r.v[r.n++] = z;
        }
        if (x->hi < y->hi) i++; else j++;
    }
    set_copy(a, &r);
}

/* a <- a union b (both sorted, disjoint); touching pieces are merged. */
static void set_or(iset *a, const iset *b) {
    ivl all[2 * MAXI];
    int n = 0, i = 0, j = 0;
    while (i < a->n || j < b->n) {
        if (j >= b->n || (i < a->n && a->v[i].lo <= b->v[j].lo)) all[n++] = a->v[i++];
        else all[n++] = b->v[j++];
    }
    iset r; r.n = 0;
    for (int k = 0; k < n; k++) {
        if (r.n > 0 && all[k].lo <= r.v[r.n - 1].hi) {
            if (all[k].hi > r.v[r.n - 1].hi) {
                r.v[r.n - 1].hi = all[k].hi; r.v[r.n - 1].fhi = all[k].fhi; r.v[r.n - 1].chi = all[k].chi;
            }
        } else {
            if (r.n >= MAXI) abort();
            r.v[r.n++] = all[k];
        }
    }
    set_copy(a, &r);
}

/* Optional record of every finite crossing computed while building a line
 * set (before intersection): used only for the error bound of the step. */
#define MAXX 256
typedef struct { int n; double t[MAXX]; int f[MAXX]; double c[MAXX]; } xrec;
static void rec_set(xrec *R, const iset *s) {
    if (!R) return;
    for (int i = 0; i < s->n; i++) {
        if (isfinite(s->v[i].lo) && R->n < MAXX) { R->t[R->n] = s->v[i].lo; R->f[R->n] = s->v[i].flo; R->c[R->n++] = s->v[i].clo; }
        if (isfinite(s->v[i].hi) && R->n < MAXX) { R->t[R->n] = s->v[i].hi; R->f[R->n] = s->v[i].fhi; R->c[R->n++] = s->v[i].chi; }
    }
}

/* { s : c + s*w <= h } (upper = 0) or { s : c + s*w >= h } (upper = 1). */
static void half_set(double c, double w, double h, int upper, int f, iset *s) {
    if (w == 0.0) {
        if (upper ? c >= h : c <= h) set_all(s); else set_empty(s);
        return;
    }
    double t = (h - c) / w;
    int below_after = (w < 0.0);           /* c + s w decreases with s */
    int keep_after = upper ? !below_after : below_after;
    if (keep_after) set_one(s, t, f, INFINITY, INFINITY, F_NONE, INFINITY);
    else set_one(s, -INFINITY, F_NONE, INFINITY, t, f, INFINITY);
}

/* { s : |c + s*w| <= h } for a slab; faces fm (at -h) and fp (at +h). */
static void slab_set(double c, double w, double h, int fm, int fp, iset *s) {
    if (w == 0.0) {
        if (fabs(c) <= h) set_all(s); else set_empty(s);
        return;
    }
    double a = (-h - c) / w;   /* where c + s w = -h */
    double b = (h - c) / w;    /* where c + s w = +h */
    if (w > 0.0) set_one(s, a, fm, INFINITY, b, fp, INFINITY);
    else         set_one(s, b, fp, INFINITY, a, fm, INFINITY);
}

/* ---- double-double arithmetic ----------------------------------------
 * Quadric coefficients, discriminants and roots are carried as unevaluated
 * sums hi + lo of two doubles (T. J. Dekker, "A floating-point technique for
 * extending the available precision", Numer. Math. 18, 1971; D. E. Knuth,
 * TAOCP vol. 2, the error-free sum; Y. Hida, X. S. Li, D. H. Bailey,
 * "Algorithms for quad-double precision floating point arithmetic", 2001).
 * With ~106 significant bits the roots are exact to FP64 rounding for the
 * given FP64 local coordinates, even next to tangency or a cone apex. */
typedef struct { double hi, lo; } dd;

static dd dd_of(double a) { dd r = { a, 0.0 }; return r; }
static dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    dd r = { s, (a - (s - bb)) + (b - bb) };
    return r;
}
static dd fast_two_sum(double a, double b) {
    double s = a + b;
    dd r = { s, b - (s - a) };
    return r;
}
static dd two_prod(double a, double b) {
    double p = a * b;
    dd r = { p, fma(a, b, -p) };
    return r;
}
static dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd a) { dd r = { -a.hi, -a.lo }; return r; }
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
static dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul(dd_of(q1), b));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul(dd_of(q2), b));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add(q, dd_of(q3));
}
static dd dd_sqrt(dd a) {
    if (a.hi <= 0.0) return dd_of(0.0);
    double x = sqrt(a.hi);
    /* one Newton step on x^2 = a in double-double */
    dd e = dd_sub(a, two_prod(x, x));
    return dd_add(dd_of(x), dd_of(e.hi / (2.0 * x)));
}
static int dd_sign(dd a) { return a.hi > 0.0 ? 1 : (a.hi < 0.0 ? -1 : (a.lo > 0.0 ? 1 : (a.lo < 0.0 ? -1 : 0))); }
static double dd_val(dd a) { return a.hi + a.lo; }


/* { s : A s^2 + 2 B s + C <= 0 }, endpoints tagged with surface f;
 * coefficients in double-double. */
static void quad_le0(dd A, dd B, dd C, int f, iset *s) {
    int sa = dd_sign(A), sb = dd_sign(B);
    if (sa == 0) {
        if (sb == 0) {
            if (dd_sign(C) <= 0) set_all(s); else set_empty(s);
            return;
        }
        double r = dd_val(dd_div(dd_neg(C), dd_add(B, B)));
        if (sb > 0) set_one(s, -INFINITY, F_NONE, INFINITY, r, f, INFINITY);
        else        set_one(s, r, f, INFINITY, INFINITY, F_NONE, INFINITY);
        return;
    }
    dd D = dd_sub(dd_mul(B, B), dd_mul(A, C));
    if (dd_sign(D) < 0) {
        if (sa > 0) set_empty(s); else set_all(s);
        return;
    }
    dd sq = dd_sqrt(D);
    double half = dd_val(sq) / fabs(dd_val(A));
    /* q = -(B + sign(B) sqrt(D)): no cancellation; roots q/A and C/q */
    dd q = dd_neg(sb >= 0 ? dd_add(B, sq) : dd_sub(B, sq));
    double r1, r2;
    if (dd_sign(q) == 0) { r1 = 0.0; r2 = 0.0; }
    else { r1 = dd_val(dd_div(q, A)); r2 = dd_val(dd_div(C, q)); }
    double lo = r1 < r2 ? r1 : r2;
    double hi = r1 < r2 ? r2 : r1;
    if (sa > 0) {
        set_one(s, lo, f, half, hi, f, half);
    } else if (!(lo < hi)) {
        set_all(s);          /* double root of a downward parabola: <= 0 everywhere */
    } else {
        s->n = 2;
        s->v[0].lo = -INFINITY; s->v[0].flo = F_NONE; s->v[0].clo = INFINITY;
        s->v[0].hi = lo; s->v[0].fhi = f; s->v[0].chi = half;
        s->v[1].lo = hi; s->v[1].flo = f; s->v[1].clo = half;
        s->v[1].hi = INFINITY; s->v[1].fhi = F_NONE; s->v[1].chi = INFINITY;
    }
}

/* Cone radius line R(z) = a + b z through (r1 at -dz) and (r2 at +dz). */
static void cone_line(double dz, double r1, double r2, dd *a, dd *b) {
    dd sum = two_sum(r1, r2);
    a->hi = 0.5 * sum.hi; a->lo = 0.5 * sum.lo;
    *b = dd_div(two_sum(r2, -r1), dd_of(2.0 * dz));
}

/* Wedge of a tube segment: the half-plane normals, whether the wedge is the
 * intersection of the two half-planes (dphi <= pi) and whether it is all of
 * the plane (dphi >= 2 pi). */
#define ORC_PI 3.14159265358979323846
typedef struct { double n1[2], n2[2]; int convex, full, half; } wedge;
static wedge wedge_at(double sphi, double dphi) {
    wedge w;
    double f1 = sphi, f2 = sphi + dphi;
    w.n1[0] = -sin(f1); w.n1[1] = cos(f1);
    w.n2[0] = sin(f2);  w.n2[1] = -cos(f2);
    w.convex = dphi <= ORC_PI;
    w.full = !(dphi < 2.0 * ORC_PI);
    w.half = dphi == ORC_PI;
    return w;
}
/* the wedge of a tube segment (p[3], p[4]) or of a polycone (p[0], p[1]) */
static wedge wedge_of(int kind, const double *p) {
    return kind == K_PCON ? wedge_at(p[0], p[1]) : wedge_at(p[3], p[4]);
}
static int wedge_has(const wedge *w, double x, double y) {
    if (w->full) return 1;
    int a = w->n1[0] * x + w->n1[1] * y >= 0.0, b = w->n2[0] * x + w->n2[1] * y >= 0.0;
    return w->convex ? (a && b) : (a || b);
}

/* S <- S intersect the wedge w: each half-plane n.(x + s u) >= 0 is a
 * half-line of s; the wedge is their intersection or union. */
static void and_wedge(const wedge *w, const double *x, const double *u, iset *S, xrec *R) {
    if (w->full) return;
    iset t, h2;
    half_set(w->n1[0] * x[0] + w->n1[1] * x[1], w->n1[0] * u[0] + w->n1[1] * u[1], 0.0, 1, F_PHI1, &t);
    rec_set(R, &t);
    half_set(w->n2[0] * x[0] + w->n2[1] * x[1], w->n2[0] * u[0] + w->n2[1] * u[1], 0.0, 1, F_PHI2, &h2);
    rec_set(R, &h2);
    if (w->convex) set_and(&t, &h2); else set_or(&t, &h2);
    set_and(S, &t);
    /* dphi = pi: the two planes coincide, and a phi endpoint lies on the
     * face on whose side of the axis it is */
    for (int i = 0; i < S->n && w->half; i++) {
        for (int e = 0; e < 2; e++) {
            int *f = e ? &S->v[i].fhi : &S->v[i].flo;
            double tt = e ? S->v[i].hi : S->v[i].lo;
            if ((*f != F_PHI1 && *f != F_PHI2) || !isfinite(tt)) continue;
            double px = x[0] + tt * u[0], py = x[1] + tt * u[1];
            *f = (w->n1[1] * px - w->n1[0] * py >= 0.0) ? F_PHI1 : F_PHI2;
        }
    }
}

/* Coefficients of rho^2 - R(z)^2 along the line, R the radius line through
 * (r0 at z0) and (r1 at z1): R(z(s)) = R0 + Rs s with z(s) = x_z + s u_z. */
static void radius_quad(double z0, double z1, double r0, double r1, const double *x, const double *u,
                        dd A, dd B, dd C, dd *Aq, dd *Bq, dd *Cq) {
    dd b = dd_div(two_sum(r1, -r0), two_sum(z1, -z0));
    dd R0 = dd_add(dd_of(r0), dd_mul(b, two_sum(x[2], -z0)));
    dd Rs = dd_mul(b, dd_of(u[2]));
    *Aq = dd_sub(A, dd_mul(Rs, Rs));
    *Bq = dd_sub(B, dd_mul(R0, Rs));
    *Cq = dd_sub(C, dd_mul(R0, R0));
}

/* { s : za <= x_z + s u_z <= zb }.  A plane z = c is crossed at
 * (c - x_z) / u_z, the expression half_set uses as well, so that two
 * sections sharing a plane meet at the same s. */
static void zslab(const double *x, const double *u, double za, double zb, int fa, int fb, iset *s) {
    if (u[2] == 0.0) {
        if (x[2] >= za && x[2] <= zb) set_all(s); else set_empty(s);
        return;
    }
    double ta = (za - x[2]) / u[2], tb = (zb - x[2]) / u[2];
    if (u[2] > 0.0) set_one(s, ta, fa, INFINITY, tb, fb, INFINITY);
    else set_one(s, tb, fb, INFINITY, ta, fa, INFINITY);
}

/* Polycone: the union over sections of slab AND rho <= Rout(z) AND
 * rho >= Rin(z), then cut to the wedge.  Inner planes carry no face tag
 * (they are no surface); the end planes are -z (4) and +z (5). */
static void pcon_line_set(const double *p, const double *x, const double *u, dd A, dd B, dd C,
                          iset *S, xrec *R) {
    const int nz = (int)p[2];
    const double *z = p + 3, *rn = z + nz, *rx = rn + nz;
    iset sec, t, hs;
    set_empty(S);
    for (int k = 0; k + 1 < nz; k++) {
        const int fa = k == 0 ? F_ZM : F_NONE, fb = k + 2 == nz ? F_ZP : F_NONE;
        dd Aq, Bq, Cq;
        zslab(x, u, z[k], z[k + 1], fa, fb, &sec); rec_set(R, &sec);
        radius_quad(z[k], z[k + 1], rx[k], rx[k + 1], x, u, A, B, C, &Aq, &Bq, &Cq);
        quad_le0(Aq, Bq, Cq, F_SEC + 2 * k, &t); rec_set(R, &t); set_and(&sec, &t);
        if (rn[k] > 0.0 || rn[k + 1] > 0.0) {
            /* rho >= Rin(z), squared (exact on the slab, where Rin >= 0);
             * an inner radius of 0 adds its whole plane, as for the cone */
            radius_quad(z[k], z[k + 1], rn[k], rn[k + 1], x, u, A, B, C, &Aq, &Bq, &Cq);
            quad_le0(dd_neg(Aq), dd_neg(Bq), dd_neg(Cq), F_SEC + 2 * k + 1, &t); rec_set(R, &t);
            if (rn[k] == 0.0) { half_set(x[2], u[2], z[k], 0, fa, &hs); set_or(&t, &hs); }
            if (rn[k + 1] == 0.0) { half_set(x[2], u[2], z[k + 1], 1, fb, &hs); set_or(&t, &hs); }
            set_and(&sec, &t);
        }
        set_or(S, &sec);
    }
    wedge w = wedge_at(p[0], p[1]);
    and_wedge(&w, x, u, S, R);
}

/* The exact line set S for a solid in its local frame. */
static void line_set_rec(int kind, const double *p, const double *x, const double *u, iset *S, xrec *R) {
    iset t;
    if (kind == K_BOX) {
        slab_set(x[0], u[0], p[0], 0, 1, S); rec_set(R, S);
        slab_set(x[1], u[1], p[1], 2, 3, &t); rec_set(R, &t); set_and(S, &t);
        slab_set(x[2], u[2], p[2], 4, 5, &t); rec_set(R, &t); set_and(S, &t);
        return;
    }
    /* rho^2(s) = A s^2 + 2 B s + C, exactly in double-double */
    dd A = dd_add(two_prod(u[0], u[0]), two_prod(u[1], u[1]));
    dd B = dd_add(two_prod(x[0], u[0]), two_prod(x[1], u[1]));
    dd C = dd_add(two_prod(x[0], x[0]), two_prod(x[1], x[1]));
    if (kind == K_PCON) {
        pcon_line_set(p, x, u, A, B, C, S, R);
        return;
    }
    if (kind == K_TUBE || kind == K_TUBS) {
        double rmin = p[0], rmax = p[1], dz = p[2];
        slab_set(x[2], u[2], dz, F_ZM, F_ZP, S); rec_set(R, S);
        quad_le0(A, B, dd_sub(C, two_prod(rmax, rmax)), F_OUT, &t); rec_set(R, &t); set_and(S, &t);
        if (rmin > 0.0) {
            /* rho^2 >= rmin^2  <=>  -(rho^2 - rmin^2) <= 0 */
            dd Ci = dd_sub(C, two_prod(rmin, rmin));
            quad_le0(dd_neg(A), dd_neg(B), dd_neg(Ci), F_IN, &t); rec_set(R, &t); set_and(S, &t);
        }
        if (kind == K_TUBS) {
            wedge w = wedge_of(kind, p);
            and_wedge(&w, x, u, S, R);
        }
        return;
    }
    /* cone: rho <= Rmax(z) and rho >= Rmin(z) inside |z| <= dz; both radius
     * lines are non-negative on the slab, so squaring is exact as a set
     * statement there. */
    double dz = p[0];
    dd a, b;
    slab_set(x[2], u[2], dz, F_ZM, F_ZP, S); rec_set(R, S);
    cone_line(dz, p[2], p[4], &a, &b);
    {
        dd R0 = dd_add(a, dd_mul(b, dd_of(x[2]))), Rs = dd_mul(b, dd_of(u[2]));
        quad_le0(dd_sub(A, dd_mul(Rs, Rs)), dd_sub(B, dd_mul(R0, Rs)), dd_sub(C, dd_mul(R0, R0)), F_OUT, &t);
        rec_set(R, &t); set_and(S, &t);
    }
    if (p[1] > 0.0 || p[3] > 0.0) {
        /* rho >= Rmin(z).  Squared, this is exact on the slab (Rmin >= 0
         * there); where an inner radius is 0 the condition also holds on the
         * whole end plane through that apex, which is added explicitly: the
         * squared form alone is degenerate at the apex. */
        cone_line(dz, p[1], p[3], &a, &b);
        dd R0 = dd_add(a, dd_mul(b, dd_of(x[2]))), Rs = dd_mul(b, dd_of(u[2]));
        dd Ai = dd_sub(A, dd_mul(Rs, Rs)), Bi = dd_sub(B, dd_mul(R0, Rs)), Ci = dd_sub(C, dd_mul(R0, R0));
        quad_le0(dd_neg(Ai), dd_neg(Bi), dd_neg(Ci), F_IN, &t); rec_set(R, &t);
        iset hs;
        if (p[1] == 0.0) { half_set(x[2], u[2], -dz, 0, F_ZM, &hs); set_or(&t, &hs); }
        if (p[3] == 0.0) { half_set(x[2], u[2], dz, 1, F_ZP, &hs); set_or(&t, &hs); }
        set_and(S, &t);
    }
}

static void line_set(int kind, const double *p, const double *x, const double *u, iset *S) {
    line_set_rec(kind, p, x, u, S, NULL);
}

typedef struct { double s; int face; double chord; } hitinfo;

static hitinfo dist_out_info(int kind, const double *p, const double *x, const double *u) {
    iset S; line_set(kind, p, x, u, &S);
    hitinfo h = { INFINITY, F_NONE, INFINITY };
    for (int i = 0; i < S.n; i++) {
        if (S.v[i].hi >= 0.0) {
            if (S.v[i].lo > 0.0) { h.s = S.v[i].lo; h.face = S.v[i].flo; h.chord = S.v[i].clo; }
            else { h.s = 0.0; h.face = F_NONE; h.chord = INFINITY; }
            return h;
        }
    }
    return h;
}

/* Re-entry into a solid the track has just left (its start point is on the
 * solid's surface): the first component of S that begins after s = 0; the
 * component holding (or ending at) the start point is the one just left. */
static hitinfo dist_reentry_info(int kind, const double *p, const double *x, const double *u) {
    iset S; line_set(kind, p, x, u, &S);
    hitinfo h = { INFINITY, F_NONE, INFINITY };
    for (int i = 0; i < S.n; i++) {
        if (S.v[i].lo > 0.0) { h.s = S.v[i].lo; h.face = S.v[i].flo; h.chord = S.v[i].clo; return h; }
    }
    return h;
}

/* Exit from a solid the track has just entered through its surface (its
 * start point lies on that surface, inside or a rounding outside): the end
 * of the first component of S that ends after s = 0; 0 if there is none. */
static hitinfo dist_in_entered_info(int kind, const double *p, const double *x, const double *u) {
    iset S; line_set(kind, p, x, u, &S);
    hitinfo h = { 0.0, F_NONE, INFINITY };
    for (int i = 0; i < S.n; i++) {
        if (S.v[i].hi > 0.0) { h.s = S.v[i].hi; h.face = S.v[i].fhi; h.chord = S.v[i].chi; return h; }
    }
    return h;
}

static hitinfo dist_in_info(int kind, const double *p, const double *x, const double *u) {
    iset S; line_set(kind, p, x, u, &S);
    hitinfo h = { 0.0, F_NONE, INFINITY };
    for (int i = 0; i < S.n; i++) {
        if (S.v[i].lo <= 0.0 && S.v[i].hi >= 0.0) {
            h.s = S.v[i].hi; h.face = S.v[i].fhi; h.chord = S.v[i].chi;
            return h;
        }
    }
    return h;
}

double orc_dist_out(int kind, const double *p, const double *x, const double *u) {
    return dist_out_info(kind, p, x, u).s;
}
double orc_dist_in(int kind, const double *p, const double *x, const double *u) {
    return dist_in_info(kind, p, x, u).s;
}

/* (r, z) in the polycone's cross-section (the meridian half-plane, r >= 0):
 * in some section whose z-range holds z, between its interpolated radii. */
static int pcon_in2(const double *p, double r, double z0) {
    const int nz = (int)p[2];
    const double *z = p + 3, *rn = z + nz, *rx = rn + nz;
    if (!(r >= 0.0)) return 0;
    double r2 = r * r;
    for (int k = 0; k + 1 < nz; k++) {
        if (!(z0 >= z[k] && z0 <= z[k + 1])) continue;
        double f = (z0 - z[k]) / (z[k + 1] - z[k]);
        double rmin = rn[k] + (rn[k + 1] - rn[k]) * f;
        double rmax = rx[k] + (rx[k + 1] - rx[k]) * f;
        if (r2 <= rmax * rmax && r2 >= rmin * rmin) return 1;
    }
    return 0;
}

/* Closed-solid membership, straight from the definitions. */
int orc_contains(int kind, const double *p, const double *x) {
    if (kind == K_BOX)
        return fabs(x[0]) <= p[0] && fabs(x[1]) <= p[1] && fabs(x[2]) <= p[2];
    double r2 = x[0] * x[0] + x[1] * x[1];
    if (kind == K_PCON) {
        if (!pcon_in2(p, sqrt(r2), x[2])) return 0;
        wedge w = wedge_of(kind, p);
        return wedge_has(&w, x[0], x[1]);
    }
    if (kind == K_TUBE || kind == K_TUBS) {
        if (fabs(x[2]) > p[2]) return 0;
        if (!(r2 <= p[1] * p[1] && r2 >= p[0] * p[0])) return 0;
        if (kind == K_TUBE) return 1;
        wedge w = wedge_of(kind, p);
        return wedge_has(&w, x[0], x[1]);
    }
    double dz = p[0];
    if (fabs(x[2]) > dz) return 0;
    double f = (x[2] + dz) / (2.0 * dz);
    double rmin = p[1] + (p[3] - p[1]) * f;
    double rmax = p[2] + (p[4] - p[2]) * f;
    return r2 <= rmax * rmax && r2 >= rmin * rmin;
}

/* Euclidean distance from (px,pz) to the segment (ax,az)-(bx,bz). */
static double seg_dist(double px, double pz, double ax, double az, double bx, double bz) {
    double ex = bx - ax, ez = bz - az;
    double wx = px - ax, wz = pz - az;
    double L2 = ex * ex + ez * ez;
    double t = 0.0;
    if (L2 > 0.0) {
        t = (wx * ex + wz * ez) / L2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    double cx = ax + t * ex - px, cz = az + t * ez - pz;
    return sqrt(cx * cx + cz * cz);
}

/* 2-D distance from (r, z) to the boundary edges of the polycone's
 * cross-section: the two end caps, the outer edge of every section, and
 * its inner edge unless that lies on the axis (both inner radii 0) and
 * axis == 0. */
static double pcon_edges(const double *p, double r, double z0, int axis) {
    const int nz = (int)p[2];
    const double *z = p + 3, *rn = z + nz, *rx = rn + nz;
    double d = seg_dist(r, z0, rn[0], z[0], rx[0], z[0]);
    double e = seg_dist(r, z0, rn[nz - 1], z[nz - 1], rx[nz - 1], z[nz - 1]);
    if (e < d) d = e;
    for (int k = 0; k + 1 < nz; k++) {
        e = seg_dist(r, z0, rx[k], z[k], rx[k + 1], z[k + 1]);
        if (e < d) d = e;
        if (axis || rn[k] > 0.0 || rn[k + 1] > 0.0) {
            e = seg_dist(r, z0, rn[k], z[k], rn[k + 1], z[k + 1]);
            if (e < d) d = e;
        }
    }
    return d;
}

/* Safety: exact distance to the nearest boundary point.  inside=1 gives the
 * distance for a point inside the solid, inside=0 for a point outside
 * (0 when the point is in fact on the other side). */
double orc_safety(int kind, const double *p, const double *x, int inside) {
    int in = orc_contains(kind, p, x);
    if (inside != in) return 0.0;
    if (kind == K_BOX) {
        if (in) {
            double s = p[0] - fabs(x[0]);
            double s1 = p[1] - fabs(x[1]), s2 = p[2] - fabs(x[2]);
            if (s1 < s) s = s1;
            if (s2 < s) s = s2;
            return s;
        }
        double a = fabs(x[0]) - p[0], b = fabs(x[1]) - p[1], c = fabs(x[2]) - p[2];
        if (a < 0.0) a = 0.0;
        if (b < 0.0) b = 0.0;
        if (c < 0.0) c = 0.0;
        return sqrt(a * a + b * b + c * c);
    }
    if (kind == K_PCON) {
        wedge w = wedge_of(kind, p);
        double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
        /* distance to a phi face: its plane's normal distance h, and the 2-D
         * distance of the point's projection (r along the face's direction,
         * z) to the cross-section */
        double face[2] = { INFINITY, INFINITY };
        if (!w.full) {
            double e1[2] = { w.n1[1], -w.n1[0] }, e2[2] = { -w.n2[1], w.n2[0] };
            for (int i = 0; i < 2; i++) {
                const double *n = i ? w.n2 : w.n1, *e = i ? e2 : e1;
                double h = n[0] * x[0] + n[1] * x[1];
                double r = e[0] * x[0] + e[1] * x[1];
                double d2 = pcon_in2(p, r, x[2]) ? 0.0 : pcon_edges(p, r, x[2], 1);
                face[i] = sqrt(h * h + d2 * d2);
            }
        }
        if (in) {
            /* the edges of the cross-section other than those on the axis
             * (inside a whole turn the axis is no surface; with a wedge the
             * phi faces hold it) */
            double d = pcon_edges(p, rho, x[2], 0);
            if (face[0] < d) d = face[0];
            if (face[1] < d) d = face[1];
            return d;
        }
        /* azimuth in the wedge: the 2-D distance to the cross-section in
         * the point's meridian half-plane; outside it: a phi face (for every
         * radius and height the nearest azimuth of the wedge is an end) */
        if (w.full || wedge_has(&w, x[0], x[1])) return pcon_edges(p, rho, x[2], 1);
        return face[0] < face[1] ? face[0] : face[1];
    }
    if (kind == K_TUBS) {
        wedge w = wedge_of(kind, p);
        double rmin = p[0], rmax = p[1], dz = p[2];
        double rho = sqrt(x[0] * x[0] + x[1] * x[1]), az = fabs(x[2]);
        /* distance to the phi face at unit direction e (the rectangle
         * rmin <= r <= rmax, |z| <= dz of its half-plane) */
        double e1[2] = { w.n1[1], -w.n1[0] }, e2[2] = { -w.n2[1], w.n2[0] };
        double face[2];
        for (int i = 0; i < 2; i++) {
            const double *n = i ? w.n2 : w.n1, *e = i ? e2 : e1;
            double h = n[0] * x[0] + n[1] * x[1];
            double r = e[0] * x[0] + e[1] * x[1];
            double rc = r < rmin ? rmin : (r > rmax ? rmax : r);
            double zc = az > dz ? az - dz : 0.0;
            face[i] = sqrt(h * h + (r - rc) * (r - rc) + zc * zc);
        }
        if (in) {
            double d = rmax - rho;
            if (dz - az < d) d = dz - az;
            if (rmin > 0.0 && rho - rmin < d) d = rho - rmin;
            if (!w.full) {
                if (face[0] < d) d = face[0];
                if (face[1] < d) d = face[1];
            }
            return d;
        }
        if (w.full || wedge_has(&w, x[0], x[1])) {
            /* azimuth inside the wedge: the tube's own 2-D distance */
            double dr = rho > rmax ? rho - rmax : (rho < rmin ? rmin - rho : 0.0);
            double dzo = az > dz ? az - dz : 0.0;
            return sqrt(dr * dr + dzo * dzo);
        }
        /* azimuth outside: for every radius and height the nearest azimuth
         * of the wedge is one of its ends, so a phi face is nearest */
        return face[0] < face[1] ? face[0] : face[1];
    }
    /* Solids of revolution: the distance is the 2-D distance in the meridian
     * half-plane (rho, z) to the cross-section polygon
     * (rmin1,-dz) (rmax1,-dz) (rmax2,dz) (rmin2,dz). */
    double dz, rmin1, rmax1, rmin2, rmax2;
    if (kind == K_TUBE) { rmin1 = rmin2 = p[0]; rmax1 = rmax2 = p[1]; dz = p[2]; }
    else { dz = p[0]; rmin1 = p[1]; rmax1 = p[2]; rmin2 = p[3]; rmax2 = p[4]; }
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]), z = x[2];
    double d = seg_dist(rho, z, rmin1, -dz, rmax1, -dz);
    double e = seg_dist(rho, z, rmax1, -dz, rmax2, dz);  if (e < d) d = e;
    e = seg_dist(rho, z, rmax2, dz, rmin2, dz);          if (e < d) d = e;
    /* the edge on the axis is no surface when both inner radii are 0 */
    if (!in || rmin1 > 0.0 || rmin2 > 0.0) {
        e = seg_dist(rho, z, rmin2, dz, rmin1, -dz);     if (e < d) d = e;
    }
    return d;
}

/* Gradient g = grad_x F of the winning surface F(x; theta) = 0 at the local
 * point xs (F > 0 outside the solid) and dF/dtheta for the five shape
 * parameters.  Faces as tagged by line_set. */
static void surface_grad(int kind, const double *p, int f, const double *xs, double *g, double *dF) {
    for (int k = 0; k < 3; k++) g[k] = 0.0;
    for (int k = 0; k < 5; k++) dF[k] = 0.0;
    if (kind == K_BOX) {
        int ax = f / 2; double sg = (f % 2) ? 1.0 : -1.0;
        g[ax] = sg;                  /* F = sg*x_ax - h_ax */
        dF[ax] = -1.0;
        return;
    }
    if (f == F_PHI1 || f == F_PHI2) {
        /* F = -n.(x, y) for the face's normal n; theta = (..., sphi, dphi),
         * the row slots 3, 4 of a tube segment and 0, 1 of a polycone */
        wedge w = wedge_of(kind, p);
        const int is = kind == K_PCON ? 0 : 3;
        if (f == F_PHI1) {
            g[0] = -w.n1[0]; g[1] = -w.n1[1];
            dF[is] = w.n1[1] * xs[0] - w.n1[0] * xs[1];          /* e1 . (x, y) */
        } else {
            g[0] = -w.n2[0]; g[1] = -w.n2[1];
            double de = -(-w.n2[1] * xs[0] + w.n2[0] * xs[1]);  /* -e2 . (x, y) */
            dF[is] = de; dF[is + 1] = de;
        }
        return;
    }
    if (kind == K_PCON) {
        /* end planes F = z[0] - z, z - z[nz-1]; section surfaces F = +-(rho^2
         * - R(z)^2).  The plane table gets no gradient (dF = 0). */
        const int nz = (int)p[2];
        const double *z = p + 3, *rn = z + nz, *rx = rn + nz;
        if (f == F_ZM || f == F_ZP) { g[2] = f == F_ZP ? 1.0 : -1.0; return; }
        if (f < F_SEC) return;
        const int k = (f - F_SEC) / 2, outer = ((f - F_SEC) % 2) == 0;
        const double *r = outer ? rx : rn;
        double b = (r[k + 1] - r[k]) / (z[k + 1] - z[k]);
        double Rz = r[k] + b * (xs[2] - z[k]);
        double sg = outer ? 1.0 : -1.0;
        g[0] = sg * 2.0 * xs[0]; g[1] = sg * 2.0 * xs[1]; g[2] = sg * (-2.0 * Rz * b);
        return;
    }
    int tubelike = kind == K_TUBE || kind == K_TUBS;
    double dz = tubelike ? p[2] : p[0];
    int dzi = tubelike ? 2 : 0;
    if (f == F_ZM || f == F_ZP) {
        double sg = (f == F_ZP) ? 1.0 : -1.0;
        g[2] = sg; dF[dzi] = -1.0;   /* F = sg*z - dz */
    } else if (tubelike) {
        double r = (f == F_OUT) ? p[1] : p[0];
        double sg = (f == F_OUT) ? 1.0 : -1.0;   /* outside of the solid is F > 0 */
        g[0] = sg * 2.0 * xs[0]; g[1] = sg * 2.0 * xs[1];
        dF[(f == F_OUT) ? 1 : 0] = sg * (-2.0 * r);
    } else {
        int outer = (f == F_OUT);
        double r1 = outer ? p[2] : p[1], r2 = outer ? p[4] : p[3];
        double sg = outer ? 1.0 : -1.0;
        double w2 = (xs[2] + dz) / (2.0 * dz);    /* weight of r2 */
        double Rz = r1 + (r2 - r1) * w2;
        double dRdz = (r2 - r1) / (2.0 * dz);
        /* F = sg (x^2 + y^2 - R(z)^2) */
        g[0] = sg * 2.0 * xs[0]; g[1] = sg * 2.0 * xs[1];
        g[2] = sg * (-2.0 * Rz * dRdz);
        double dRdr1 = 1.0 - w2, dRdr2 = w2;
        /* dR/d(dz) at fixed z: w2 = (z+dz)/(2dz) -> dw2/ddz = -z/(2 dz^2) */
        double dRddz = (r2 - r1) * (-xs[2] / (2.0 * dz * dz));
        dF[outer ? 2 : 1] = sg * (-2.0 * Rz * dRdr1);
        dF[outer ? 4 : 3] = sg * (-2.0 * Rz * dRdr2);
        dF[0] = sg * (-2.0 * Rz * dRddz);
    }
}

/* ------------------------------------------------------------------ */
/* the navigator (Fig. 1)                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int mkind; const double *mparams;
    int nd; const int32_t *kinds; const double *params, *rot, *trans;
    const double *pdata;   /* polycone plane table */
} orc_scene;

/* Parameter block of a solid as the shape routines read it: its row of five,
 * or for a polycone [sphi, dphi, nz, z[nz], rmin[nz], rmax[nz]] gathered
 * from the plane table (row = (sphi, dphi, nz, offset, 0); the table holds
 * at the offset nz z-values, then the nz inner, then the nz outer radii). */
#define PBUF (3 + 3 * MAXZ)
static const double *shape_block(int kind, const double *row, const double *pdata, double *buf) {
    if (kind != K_PCON) return row;
    const int nz = (int)row[2];
    const int64_t off = (int64_t)row[3];
    if (nz < 2 || nz > MAXZ || off < 0 || !pdata) abort();
    buf[0] = row[0]; buf[1] = row[1]; buf[2] = row[2];
    memcpy(buf + 3, pdata + off, (size_t)(3 * nz) * sizeof(double));
    return buf;
}
#define MOTHER(sc, buf) shape_block((sc)->mkind, (sc)->mparams, (sc)->pdata, buf)
#define DAUGHTER(sc, j, buf) shape_block((sc)->kinds[j], (sc)->params + 5 * (j), (sc)->pdata, buf)

/* x = R^T (p - t), u = R^T d: master -> local (Sec. 3.1). */
static void to_local(const orc_scene *sc, int j, const double *pw, const double *dw,
                     double *x, double *u) {
    const double *R = sc->rot + 9 * j, *t = sc->trans + 3 * j;
    double w0 = pw[0] - t[0], w1 = pw[1] - t[1], w2 = pw[2] - t[2];
    for (int k = 0; k < 3; k++) {
        x[k] = R[0 + k] * w0 + R[3 + k] * w1 + R[6 + k] * w2;
        u[k] = R[0 + k] * dw[0] + R[3 + k] * dw[1] + R[6 + k] * dw[2];
    }
}

static int bad_input(const double *pw, const double *dw) {
    for (int k = 0; k < 3; k++)
        if (!isfinite(pw[k]) || !isfinite(dw[k])) return 1;
    return dw[0] == 0.0 && dw[1] == 0.0 && dw[2] == 0.0;
}

static double shape_scale(int kind, const double *p) {
    if (kind == K_BOX) { double m = p[0]; if (p[1] > m) m = p[1]; if (p[2] > m) m = p[2]; return m; }
    if (kind == K_PCON) {
        const int nz = (int)p[2];
        double m = 0.0;
        for (int k = 0; k < nz; k++) {
            if (fabs(p[3 + k]) > m) m = fabs(p[3 + k]);
            if (p[3 + 2 * nz + k] > m) m = p[3 + 2 * nz + k];
        }
        return m;
    }
    if (kind == K_TUBE || kind == K_TUBS) return p[1] > p[2] ? p[1] : p[2];
    double m = p[0]; if (p[2] > m) m = p[2]; if (p[4] > m) m = p[4]; return m;
}

typedef struct {
    double step;   int hit;
    double second; /* second-smallest candidate (mother included)              */
    int face;      /* surface of the winner                                   */
    double err;    /* a-priori FP64 error bound of the step                      */
} navres;

/* Radius line R(z) = ra + rb z of a quadric face (rho = R(z)); 0 for a face
 * that is a plane. */
static int face_line(int kind, const double *p, int f, double *ra, double *rb) {
    if (kind == K_BOX || f == F_ZM || f == F_ZP || f == F_PHI1 || f == F_PHI2 || f < 0) return 0;
    if (kind == K_TUBE || kind == K_TUBS) {
        if (f != F_OUT && f != F_IN) return 0;
        *ra = f == F_OUT ? p[1] : p[0];
        *rb = 0.0;
        return 1;
    }
    if (kind == K_CONE) {
        if (f != F_OUT && f != F_IN) return 0;
        const double r1 = f == F_OUT ? p[2] : p[1], r2 = f == F_OUT ? p[4] : p[3];
        *rb = (r2 - r1) / (2.0 * p[0]);
        *ra = 0.5 * (r1 + r2);
        return 1;
    }
    if (f < F_SEC) return 0;
    const int nz = (int)p[2];
    const double *z = p + 3, *rn = z + nz, *rx = rn + nz;
    const int k = (f - F_SEC) / 2;
    const double *r = ((f - F_SEC) % 2) == 0 ? rx : rn;
    if (k + 1 >= nz) return 0;
    *rb = (r[k + 1] - r[k]) / (z[k + 1] - z[k]);
    *ra = r[k] - *rb * z[k];
    return 1;
}

/* blocked >= 0: that daughter was just left through its surface; it enters
 * the minimum with its re-entry distance instead of DistFromOutside (0).
 * blocked == -2: the track has just entered the mother through its surface;
 * the mother's exit is that of the component being entered, and a start
 * point a rounding outside the mother is not "outside".
 * frame: how many placements (levels of a geometry tree) were applied, in
 * FP64, to bring the track into this volume's frame, and fscale (mm) the
 * size of the coordinates they moved (0, 0 for a track given in the frame). */
/* A-priori FP64 error bound (in units of the step, |d|) of the crossing of
 * solid (kind, prm) at parameter s of its local line x + s u, for a track at
 * distance pn from the origin of the volume's frame with direction norm dn,
 * the solid placed at distance tnorm, below `frame` FP64 placement levels that
 * moved coordinates of size fscale:
 *   E = eps [ 8 ((pn + tnorm + s dn)(1 + frame) + frame fscale) cond / dn
 *             + 16 qcoef ],  eps = 2^-53,
 * over every surface crossing of the solid that coincides with s within
 * 1e-6 (1 + s) (edges, rims, apexes: which surface is crossed first is
 * decided by rounding there):
 *   cond = max(1 + L/l, 1 + |g||d|/|g.d|): a position error moves the hit by
 *     itself over |d| cos(incidence) (g the surface gradient at the hit), and
 *     a quadric root by L/l more (L the solid's size, l the half-chord);
 *   qcoef = sum|terms| / |F'(s)| of the quadric rho^2 - R(z)^2 = A s^2 +
 *     2 B s + C along the line: rounding its terms moves the root by a few eps
 *     times this (a far-away small solid: |x| >> its size), with sum|terms|
 *     <= (|x_perp| + |s||u_perp|)^2 + (|ra| + |rb| (|x_z| + |s||u_z|))^2 and
 *     |F'(s)| = |g.u|. */
static double crossing_err(int kind, const double *prm, const double *x, const double *u, double s, double pn,
                           double dn, double tnorm, int frame, double fscale) {
    double cond = 1.0, qcoef = 0.0;
    if (isfinite(s)) {
        double g[3], dF[5];
        xrec R; R.n = 0;
        iset S;
        line_set_rec(kind, prm, x, u, &S, &R);
        const double sh = shape_scale(kind, prm);
        for (int e = 0; e < R.n; e++) {
            if (!(fabs(R.t[e] - s) <= 1e-6 * (1.0 + s)) || R.f[e] == F_NONE) continue;
            const double te = R.t[e];
            const double xs[3] = { x[0] + te * u[0], x[1] + te * u[1], x[2] + te * u[2] };
            surface_grad(kind, prm, R.f[e], xs, g, dF);
            const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            const double gd = fabs(g[0] * u[0] + g[1] * u[1] + g[2] * u[2]);
            const double c2 = gd > 0.0 ? 1.0 + gn * dn / gd : INFINITY;
            if (c2 > cond) cond = c2;
            if (!isinf(R.c[e])) {
                const double c1 = 1.0 + sh / (R.c[e] * dn);
                if (c1 > cond) cond = c1;
            }
            double ra, rb;
            if (face_line(kind, prm, R.f[e], &ra, &rb)) {
                const double ate = fabs(te);
                const double m1 = sqrt(x[0] * x[0] + x[1] * x[1]) + ate * sqrt(u[0] * u[0] + u[1] * u[1]);
                const double m2 = fabs(ra) + fabs(rb) * (fabs(x[2]) + ate * fabs(u[2]));
                const double q = gd > 0.0 ? (m1 * m1 + m2 * m2) / gd : INFINITY;
                if (q > qcoef) qcoef = q;
            }
        }
    }
    const double eps = ldexp(1.0, -53);
    const double sd = isfinite(s) ? s * dn : 0.0;
    return eps * (8.0 * ((pn + tnorm + sd) * (1.0 + frame) + frame * fscale) * cond / dn + 16.0 * qcoef);
}

/* blocked >= 0: that daughter was just left through its surface; it enters
 * the minimum with its re-entry distance instead of DistFromOutside (0).
 * blocked == -2: the track has just entered the mother through its surface;
 * the mother's exit is that of the component being entered, and a start
 * point a rounding outside the mother is not "outside".
 * frame: how many placements (levels of a geometry tree) were applied, in
 * FP64, to bring the track into this volume's frame, and fscale (mm) the
 * size of the coordinates they moved (0, 0 for a track given in the frame).
 * err bounds the FP64 error of the step: the largest crossing_err() of the
 * winner and of every candidate within 1e-6 (1 + s) of it (one of those may
 * win under another rounding). */
static navres navigate_one_f(const orc_scene *sc, const double *pw, const double *dw, int blocked, int frame,
                             double fscale) {
    navres r;
    r.second = INFINITY; r.face = F_NONE; r.err = 0.0;
    const int entered = blocked == -2;
    if (bad_input(pw, dw)) { r.step = NAN; r.hit = -2; return r; }
    double mb[PBUF], db[PBUF];
    const double *mp = MOTHER(sc, mb);
    if (!entered && !orc_contains(sc->mkind, mp, pw)) { r.step = 0.0; r.hit = -2; return r; }
    hitinfo m = entered ? dist_in_entered_info(sc->mkind, mp, pw, dw)
                        : dist_in_info(sc->mkind, mp, pw, dw);
    double best = m.s;
    int hit = -1, face = m.face;
    double second = INFINITY;
    double cs[sc->nd > 0 ? sc->nd : 1];   /* every daughter's candidate step */
    for (int j = 0; j < sc->nd; j++) {
        double x[3], u[3];
        to_local(sc, j, pw, dw, x, u);
        const double *pj = DAUGHTER(sc, j, db);
        hitinfo h = j == blocked ? dist_reentry_info(sc->kinds[j], pj, x, u)
                                 : dist_out_info(sc->kinds[j], pj, x, u);
        cs[j] = h.s;
        if (h.s < best) {
            second = best;
            best = h.s; hit = j; face = h.face;
        } else if (h.s < second) {
            second = h.s;
        }
    }
    r.step = best; r.hit = hit; r.second = second; r.face = face;
    const double pn = sqrt(pw[0] * pw[0] + pw[1] * pw[1] + pw[2] * pw[2]);
    const double dn = sqrt(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
    const double win = 1e-6 * (1.0 + best);
    double err = 0.0;
    if (hit == -1 || (isfinite(best) && fabs(m.s - best) <= win)) {
        const double e = crossing_err(sc->mkind, mp, pw, dw, m.s, pn, dn, 0.0, frame, fscale);
        if (e > err) err = e;
    }
    for (int j = 0; j < sc->nd; j++) {
        if (j != hit && !(isfinite(best) && fabs(cs[j] - best) <= win)) continue;
        double x[3], u[3];
        to_local(sc, j, pw, dw, x, u);
        const double *t = sc->trans + 3 * j;
        const double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        const double e = crossing_err(sc->kinds[j], DAUGHTER(sc, j, db), x, u, cs[j], pn, dn, tn, frame, fscale);
        if (e > err) err = e;
    }
    r.err = err;
    return r;
}

static navres navigate_one_b(const orc_scene *sc, const double *pw, const double *dw, int blocked) {
    return navigate_one_f(sc, pw, dw, blocked, 0, 0.0);
}

static navres navigate_one(const orc_scene *sc, const double *pw, const double *dw) {
    return navigate_one_b(sc, pw, dw, -1);
}

static int contains_nav(const orc_scene *sc, const double *pw) {
    double buf[PBUF];
    if (!orc_contains(sc->mkind, MOTHER(sc, buf), pw)) return -2;
    for (int j = 0; j < sc->nd; j++) {
        double x[3], u[3], zero[3] = { 0, 0, 0 };
        to_local(sc, j, pw, zero, x, u);
        if (orc_contains(sc->kinds[j], DAUGHTER(sc, j, buf), x)) return j;
    }
    return -1;
}

static double safety_nav(const orc_scene *sc, const double *pw) {
    double buf[PBUF];
    const double *mp = MOTHER(sc, buf);
    if (!orc_contains(sc->mkind, mp, pw)) return 0.0;
    double s = orc_safety(sc->mkind, mp, pw, 1);
    for (int j = 0; j < sc->nd; j++) {
        double x[3], u[3], zero[3] = { 0, 0, 0 };
        to_local(sc, j, pw, zero, x, u);
        double d = orc_safety(sc->kinds[j], DAUGHTER(sc, j, buf), x, 0);
        if (d < s) s = d;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* the under-estimating safety (ROOT-style estimate)                     */
/* ------------------------------------------------------------------ */
/*
 * A cheaper safety that may under-estimate (never over-estimate) the
 * distance: every solid is replaced by a simpler bound.
 *   Mother, point inside: box and tube the exact inside distance; cone the
 *     least distance to the supporting lines of its meridian trapezoid (exact
 *     for a convex section); a whole-turn polycone whose z-range holds its
 *     origin the inside distance of its inscribed tube (radii from the
 *     largest inner to the least outer radius, half-length the nearer end
 *     plane's distance to the origin), 0 outside that tube; tube segments
 *     and other polycones 0 (no bound).
 *   Daughter, point outside: box and tube the exact distance; cone the
 *     largest signed distance to a supporting half-plane of its trapezoid
 *     (z-slab, outer radius line, and the inner radius line when both inner
 *     radii are positive), at least 0; tube segment the
 *     distance to its whole tube; polycone the distance to its enclosing tube
 *     (least inner and largest outer radius over its z-range); each of them
 *     raised to the distance to the sphere circumscribing that bound (about
 *     the box's, tube's or cone's origin, about the middle of a polycone's
 *     z-range), if larger.
 * Each is at most that solid's exact safety, so the navigator-level value
 * min(mother, daughters) is at most the exact safety.
 */
static double rect_dist(double rho, double z, double rmin, double rmax, double zlo, double zhi) {
    double dr = rho > rmax ? rho - rmax : (rho < rmin ? rmin - rho : 0.0);
    double dz = z > zhi ? z - zhi : (z < zlo ? zlo - z : 0.0);
    return sqrt(dr * dr + dz * dz);
}

static double estimate_in(int kind, const double *p, const double *x) {
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]), az = fabs(x[2]);
    double s;
    if (kind == K_BOX) {
        s = p[0] - fabs(x[0]);
        if (p[1] - fabs(x[1]) < s) s = p[1] - fabs(x[1]);
        if (p[2] - az < s) s = p[2] - az;
    } else if (kind == K_TUBE) {
        s = p[1] - rho;
        if (p[2] - az < s) s = p[2] - az;
        if (p[0] > 0.0 && rho - p[0] < s) s = rho - p[0];
    } else if (kind == K_CONE) {
        double dz = p[0];
        double bo = (p[4] - p[2]) / (2.0 * dz), bi = (p[3] - p[1]) / (2.0 * dz);
        double ro = 0.5 * (p[2] + p[4]) + bo * x[2], ri = 0.5 * (p[1] + p[3]) + bi * x[2];
        s = dz - az;
        double e = (ro - rho) / sqrt(1.0 + bo * bo);
        if (e < s) s = e;
        if (p[1] > 0.0 || p[3] > 0.0) {
            e = (rho - ri) / sqrt(1.0 + bi * bi);
            if (e < s) s = e;
        }
    } else if (kind == K_PCON && !(p[1] < 2.0 * ORC_PI)) {
        const int nz = (int)p[2];
        const double *z = p + 3, *rn = z + nz, *rx = rn + nz;
        double lo = rn[0], hi = rx[0];
        for (int k = 1; k < nz; k++) {
            if (rn[k] > lo) lo = rn[k];
            if (rx[k] < hi) hi = rx[k];
        }
        if (!(z[0] < 0.0 && z[nz - 1] > 0.0 && lo < hi)) return 0.0;
        double hz = -z[0] < z[nz - 1] ? -z[0] : z[nz - 1];
        s = hi - rho;
        if (hz - az < s) s = hz - az;
        if (lo > 0.0 && rho - lo < s) s = rho - lo;
    } else {
        s = 0.0;
    }
    return s > 0.0 ? s : 0.0;
}

/* max(bound b, distance from x to the sphere of radius R about (0, 0, zc)) */
static double with_sphere(double b, const double *x, double zc, double R) {
    double dz = x[2] - zc;
    double d = sqrt(x[0] * x[0] + x[1] * x[1] + dz * dz) - R;
    return d > b ? d : b;
}

static double estimate_out(int kind, const double *p, const double *x) {
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
    if (kind == K_BOX) {
        double a = fabs(x[0]) - p[0], b = fabs(x[1]) - p[1], c = fabs(x[2]) - p[2];
        if (a < 0.0) a = 0.0;
        if (b < 0.0) b = 0.0;
        if (c < 0.0) c = 0.0;
        return with_sphere(sqrt(a * a + b * b + c * c), x, 0.0, sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]));
    }
    if (kind == K_TUBE || kind == K_TUBS)
        return with_sphere(rect_dist(rho, x[2], p[0], p[1], -p[2], p[2]), x, 0.0, sqrt(p[1] * p[1] + p[2] * p[2]));
    if (kind == K_PCON) {
        const int nz = (int)p[2];
        const double *z = p + 3, *rn = z + nz, *rx = rn + nz;
        double lo = rn[0], hi = rx[0];
        for (int k = 1; k < nz; k++) {
            if (rn[k] < lo) lo = rn[k];
            if (rx[k] > hi) hi = rx[k];
        }
        double hz = 0.5 * (z[nz - 1] - z[0]);
        return with_sphere(rect_dist(rho, x[2], lo, hi, z[0], z[nz - 1]), x, 0.5 * (z[0] + z[nz - 1]),
                           sqrt(hi * hi + hz * hz));
    }
    double dz = p[0];
    double bo = (p[4] - p[2]) / (2.0 * dz), bi = (p[3] - p[1]) / (2.0 * dz);
    double ro = 0.5 * (p[2] + p[4]) + bo * x[2], ri = 0.5 * (p[1] + p[3]) + bi * x[2];
    double s = fabs(x[2]) - dz;
    double e = (rho - ro) / sqrt(1.0 + bo * bo);
    if (e > s) s = e;
    if (p[1] > 0.0 && p[3] > 0.0) {
        e = (ri - rho) / sqrt(1.0 + bi * bi);
        if (e > s) s = e;
    }
    double rm = p[2] > p[4] ? p[2] : p[4];
    s = with_sphere(s, x, 0.0, sqrt(rm * rm + dz * dz));
    return s > 0.0 ? s : 0.0;
}

static double safety_estimate_nav(const orc_scene *sc, const double *pw) {
    double buf[PBUF];
    const double *mp = MOTHER(sc, buf);
    if (!orc_contains(sc->mkind, mp, pw)) return 0.0;
    double s = estimate_in(sc->mkind, mp, pw);
    for (int j = 0; j < sc->nd; j++) {
        double x[3], u[3], zero[3] = { 0, 0, 0 };
        to_local(sc, j, pw, zero, x, u);
        double d = estimate_out(sc->kinds[j], DAUGHTER(sc, j, buf), x);
        if (d < s) s = d;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* adjoint of the step (implicit function rule on the winning surface)  */
/* ------------------------------------------------------------------ */

/* For the winner hitting F(x; theta) = 0 at x* = x + s u (local frame):
 *   ds/dp = -R g/den, ds/dt = +R g/den, ds/dd = -s R g/den,
 *   ds/dtheta = -(dF/dtheta)(x*)/den,   g = grad_x F(x*), den = g . u.
 * Returns 0 when the surface or denominator is undefined. */
static int adjoint_one(const orc_scene *sc, const double *pw, const double *dw,
                       double *gp, double *gd, int *jout, double *gt, double *gprm) {
    navres nr = navigate_one(sc, pw, dw);
    *jout = nr.hit;
    for (int k = 0; k < 3; k++) { gp[k] = gd[k] = gt[k] = 0.0; }
    for (int k = 0; k < 5; k++) gprm[k] = 0.0;
    if (nr.hit < -1 || nr.face == F_NONE || !isfinite(nr.step)) return 0;
    int kind; const double *p; double x[3], u[3];
    const double *R = NULL;
    double buf[PBUF];
    if (nr.hit == -1) {
        kind = sc->mkind; p = MOTHER(sc, buf);
        for (int k = 0; k < 3; k++) { x[k] = pw[k]; u[k] = dw[k]; }
    } else {
        kind = sc->kinds[nr.hit]; p = DAUGHTER(sc, nr.hit, buf);
        to_local(sc, nr.hit, pw, dw, x, u);
        R = sc->rot + 9 * nr.hit;
    }
    double s = nr.step;
    double xs[3] = { x[0] + s * u[0], x[1] + s * u[1], x[2] + s * u[2] };
    double g[3], dF[5];
    surface_grad(kind, p, nr.face, xs, g, dF);
    double den = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
    if (den == 0.0 || !isfinite(den)) return 0;
    double Rg[3];
    if (R) {
        for (int k = 0; k < 3; k++) Rg[k] = R[3 * k] * g[0] + R[3 * k + 1] * g[1] + R[3 * k + 2] * g[2];
    } else {
        Rg[0] = g[0]; Rg[1] = g[1]; Rg[2] = g[2];
    }
    for (int k = 0; k < 3; k++) {
        gp[k] = -Rg[k] / den;
        gd[k] = -s * Rg[k] / den;
        gt[k] = (nr.hit >= 0) ? Rg[k] / den : 0.0;
    }
    for (int k = 0; k < 5; k++) gprm[k] = -dF[k] / den;
    return 1;
}

/* ------------------------------------------------------------------ */
/* batch entry points (ctypes)                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_scene *sc;
    const double *px, *py, *pz, *dx, *dy, *dz;
    int64_t a, b;
    double *step, *second, *err; int32_t *hit, *face;
    double *safety; int32_t *where;
    int what;
} job;

static void *run_job(void *arg) {
    job *J = (job *)arg;
    for (int64_t i = J->a; i < J->b; i++) {
        double pw[3] = { J->px[i], J->py[i], J->pz[i] };
        if (J->what == 0) {
            double dw[3] = { J->dx[i], J->dy[i], J->dz[i] };
            navres r = navigate_one(J->sc, pw, dw);
            J->step[i] = r.step; J->hit[i] = r.hit;
            if (J->second) J->second[i] = r.second;
            if (J->err) J->err[i] = r.err;
            if (J->face) J->face[i] = r.face;
        } else if (J->what == 1) {
            J->where[i] = contains_nav(J->sc, pw);
        } else if (J->what == 2) {
            J->safety[i] = safety_nav(J->sc, pw);
        } else {
            J->safety[i] = safety_estimate_nav(J->sc, pw);
        }
    }
    return NULL;
}

static void run_threads(job *base, int64_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads == 1 || n < 2 * nthreads) {
        base->a = 0; base->b = n; run_job(base);
        return;
    }
    pthread_t th[256];
    job jobs[256];
    int64_t chunk = (n + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = *base;
        jobs[t].a = t * chunk;
        jobs[t].b = (t + 1) * chunk < n ? (t + 1) * chunk : n;
        if (jobs[t].a >= jobs[t].b) break;
        if (pthread_create(&th[t], NULL, run_job, &jobs[t]) != 0) { run_job(&jobs[t]); continue; }
        started = t + 1;
    }
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
}

#define SCENE_ARGS int mkind, const double *mparams, int nd, const int32_t *kinds, \
                   const double *params, const double *rot, const double *trans, const double *pdata
#define MAKE_SCENE orc_scene sc = { mkind, mparams, nd, kinds, params, rot, trans, pdata }

void orc_navigate(SCENE_ARGS, int64_t n,
                  const double *px, const double *py, const double *pz,
                  const double *dx, const double *dy, const double *dz,
                  double *step, int32_t *hit, double *second, double *err, int32_t *face,
                  int nthreads) {
    MAKE_SCENE;
    job J; memset(&J, 0, sizeof J);
    J.sc = &sc; J.px = px; J.py = py; J.pz = pz; J.dx = dx; J.dy = dy; J.dz = dz;
    J.step = step; J.hit = hit; J.second = second; J.err = err; J.face = face; J.what = 0;
    run_threads(&J, n, nthreads);
}

void orc_contains_nav(SCENE_ARGS, int64_t n, const double *px, const double *py,
                      const double *pz, int32_t *where, int nthreads) {
    MAKE_SCENE;
    job J; memset(&J, 0, sizeof J);
    J.sc = &sc; J.px = px; J.py = py; J.pz = pz; J.where = where; J.what = 1;
    run_threads(&J, n, nthreads);
}

void orc_safety_nav(SCENE_ARGS, int64_t n, const double *px, const double *py,
                    const double *pz, double *safety, int nthreads) {
    MAKE_SCENE;
    job J; memset(&J, 0, sizeof J);
    J.sc = &sc; J.px = px; J.py = py; J.pz = pz; J.safety = safety; J.what = 2;
    run_threads(&J, n, nthreads);
}

void orc_safety_estimate_nav(SCENE_ARGS, int64_t n, const double *px, const double *py,
                             const double *pz, double *safety, int nthreads) {
    MAKE_SCENE;
    job J; memset(&J, 0, sizeof J);
    J.sc = &sc; J.px = px; J.py = py; J.pz = pz; J.safety = safety; J.what = 3;
    run_threads(&J, n, nthreads);
}

/* Per-track adjoint of step(p, d): gp, gd (3n each, SoA), the winner index,
 * and that winner's ds/dt (3n) and ds/dparams (5n).  ok[i] = 0 where the
 * winning surface is undefined (inside a daughter, outside the mother). */
void orc_adjoint(SCENE_ARGS, int64_t n,
                 const double *px, const double *py, const double *pz,
                 const double *dx, const double *dy, const double *dz,
                 double *gp, double *gd, int32_t *winner, double *gt, double *gprm, int32_t *ok) {
    MAKE_SCENE;
    for (int64_t i = 0; i < n; i++) {
        double pw[3] = { px[i], py[i], pz[i] }, dw[3] = { dx[i], dy[i], dz[i] };
        double a[3], b[3], c[3], e[5];
        int j;
        ok[i] = adjoint_one(&sc, pw, dw, a, b, &j, c, e);
        winner[i] = j;
        for (int k = 0; k < 3; k++) { gp[k * n + i] = a[k]; gd[k * n + i] = b[k]; gt[k * n + i] = c[k]; }
        for (int k = 0; k < 5; k++) gprm[k * n + i] = e[k];
    }
}

/* Single-shape batch calls for the shape-level tests (row: the solid's row
 * of five; pdata: the plane table of a polycone). */
void orc_shape_batch(int kind, const double *row, const double *pdata, int64_t n, const double *x,
                     const double *u, int what, double *out, int32_t *face) {
    double buf[PBUF];
    const double *p = shape_block(kind, row, pdata, buf);
    for (int64_t i = 0; i < n; i++) {
        const double *xi = x + 3 * i, *ui = u + 3 * i;
        if (what == 0) { hitinfo h = dist_out_info(kind, p, xi, ui); out[i] = h.s; if (face) face[i] = h.face; }
        else if (what == 1) { hitinfo h = dist_in_info(kind, p, xi, ui); out[i] = h.s; if (face) face[i] = h.face; }
        else if (what == 2) out[i] = (double)orc_contains(kind, p, xi);
        else if (what == 3) out[i] = orc_safety(kind, p, xi, 0);
        else out[i] = orc_safety(kind, p, xi, 1);
    }
}

/* For the distance queries (what 0: DistFromOutside, 1: DistFromInside) of
 * one solid: the a-priori FP64 error bound of each answer (crossing_err(),
 * the solid placed at distance tnorm from the frame the query came from),
 * and the gap between the answer and the nearest crossing of another of the
 * solid's surfaces (which surface is crossed is decided by rounding when the
 * gap is within that bound: edges, rims, apexes). */
void orc_shape_batch_err(int kind, const double *row, const double *pdata, int64_t n, const double *x,
                         const double *u, int what, double tnorm, double *err, double *gap) {
    double buf[PBUF];
    const double *p = shape_block(kind, row, pdata, buf);
    for (int64_t i = 0; i < n; i++) {
        const double *xi = x + 3 * i, *ui = u + 3 * i;
        hitinfo h = what == 0 ? dist_out_info(kind, p, xi, ui) : dist_in_info(kind, p, xi, ui);
        const double pn = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
        const double dn = sqrt(ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]);
        err[i] = crossing_err(kind, p, xi, ui, h.s, pn, dn, tnorm, 0, 0.0);
        double g = INFINITY;
        if (isfinite(h.s)) {
            xrec R; R.n = 0;
            iset S;
            line_set_rec(kind, p, xi, ui, &S, &R);
            for (int e = 0; e < R.n; e++)
                if (R.f[e] != F_NONE && R.f[e] != h.face && fabs(R.t[e] - h.s) < g) g = fabs(R.t[e] - h.s);
        }
        gap[i] = g;
    }
}

/* ------------------------------------------------------------------ */
/* geometry tree: a step followed by final localisation                 */
/* ------------------------------------------------------------------ */
/*
 * The paper's navigator stops at "the next boundary and the volume hit" and
 * leaves the location of the track after the step out.  These functions
 * write out that last part for a tree of logical volumes.  Readings:
 *   - Logical volume v has a mother solid and daughters; daughter j of v is
 *     an instance of logical volume child[doff[v] + j] (whose mother solid is
 *     that daughter's solid), placed by the daughter's R, t.
 *   - A node is one placed instance (a path from the root).  Nodes are
 *     numbered breadth first: the root is 0; the children of a node get
 *     consecutive numbers in daughter order, nodes being expanded in the
 *     order they were numbered.
 *   - Locate(x in node N): the lowest-index daughter of N whose closed solid
 *     contains x becomes the new node, repeatedly; N itself when none does.
 *   - After the step of Fig. 1 in node N (boundary point b, in N's frame):
 *       hit j >= 0: the track is in child j; locate from there.
 *       hit -1: it leaves N.  Climbing: in the parent P the lowest-index
 *       daughter other than the one just left that contains b is entered
 *       (then located); else P itself if its solid contains b; else the
 *       track leaves P too and the climb goes on.  Leaving the root: -1.
 *       hit -2 (track not inside N's solid, or invalid input): node -2.
 *   - A track that has just left daughter j of its node (climbing) starts
 *     on j's surface, inside j's closed solid, so DistFromOutside(j) = 0
 *     would send it straight back.  Its next step takes for j the distance
 *     to RE-ENTER j instead: the start of the first component of
 *     { s : x + s u in j } that begins after s = 0 (+inf for a convex j;
 *     across the hole for a shell).  The state of a track is therefore
 *     (node, flag): flag j >= 0 after leaving daughter j into this node;
 *     -2 after entering this node through its surface, where the mother's
 *     exit is that of the component being entered (the end of the first
 *     component of S ending after s = 0), since the boundary point may lie
 *     a rounding outside the solid; -1 after Locate.
 *   - The local point of a node is obtained by applying the placements of
 *     its path one level after the other, from the root's frame (the frame
 *     of the tracks).
 */
typedef struct {
    int nlv;
    const int32_t *mkind; const double *mparams;                 /* per lv: kind, 5 params        */
    const int32_t *nd, *doff;                                    /* per lv: daughters, offset     */
    const int32_t *kinds; const double *params, *rot, *trans;    /* daughters, concatenated       */
    const int32_t *child;                                        /* per daughter: lv placed there */
    const double *pdata;                                         /* polycone plane table          */
    int root;
    /* node table */
    int nnodes;
    int32_t *lv, *parent, *slot, *first;
} orc_world;

static orc_scene world_scene(const orc_world *W, int v) {
    orc_scene s;
    const int o = W->doff[v];
    s.mkind = W->mkind[v]; s.mparams = W->mparams + 5 * v;
    s.nd = W->nd[v]; s.kinds = W->kinds + o; s.params = W->params + 5 * o;
    s.rot = W->rot + 9 * o; s.trans = W->trans + 3 * o;
    s.pdata = W->pdata;
    return s;
}

/* breadth-first node table; returns the node count or -1 past max_nodes */
static int world_nodes(orc_world *W, int max_nodes) {
    int n = 1, head = 0;
    W->lv[0] = W->root; W->parent[0] = -1; W->slot[0] = -1;
    while (head < n) {
        const int v = W->lv[head];
        W->first[head] = n;
        for (int j = 0; j < W->nd[v]; j++) {
            if (n >= max_nodes) return -1;
            W->lv[n] = W->child[W->doff[v] + j]; W->parent[n] = head; W->slot[n] = j;
            n++;
        }
        head++;
    }
    W->nnodes = n;
    return n;
}

/* x in the frame of child j of logical volume v: R^T (x - t) */
static void into_child(const orc_world *W, int v, int j, const double *x, double *xl, const double *u, double *ul) {
    orc_scene s = world_scene(W, v);
    double d0[3] = { 0, 0, 0 }, dd[3];
    to_local(&s, j, x, u ? u : d0, xl, dd);
    if (ul) { ul[0] = dd[0]; ul[1] = dd[1]; ul[2] = dd[2]; }
}

/* x in the frame of the parent: R x + t (placement of daughter j of v) */
static void into_parent(const orc_world *W, int v, int j, const double *x, double *xp) {
    const int o = W->doff[v] + j;
    const double *R = W->rot + 9 * o, *t = W->trans + 3 * o;
    for (int k = 0; k < 3; k++) xp[k] = R[3 * k] * x[0] + R[3 * k + 1] * x[1] + R[3 * k + 2] * x[2] + t[k];
}

static int descend(const orc_world *W, int node, const double *x0) {
    double x[3] = { x0[0], x0[1], x0[2] };
    for (;;) {
        const int v = W->lv[node];
        int next = -1;
        double xn[3];
        for (int j = 0; j < W->nd[v] && next < 0; j++) {
            double xl[3];
            into_child(W, v, j, x, xl, NULL, NULL);
            double buf[PBUF];
            const int o = W->doff[v] + j;
            if (orc_contains(W->kinds[o], shape_block(W->kinds[o], W->params + 5 * o, W->pdata, buf), xl)) {
                next = W->first[node] + j;
                xn[0] = xl[0]; xn[1] = xl[1]; xn[2] = xl[2];
            }
        }
        if (next < 0) return node;
        node = next;
        x[0] = xn[0]; x[1] = xn[1]; x[2] = xn[2];
    }
}

/* world point and direction in the frame of node */
static void node_frame(const orc_world *W, int node, const double *pw, const double *dw, double *x, double *u) {
    int path[64], depth = 0;
    for (int m = node; m > 0 && depth < 64; m = W->parent[m]) path[depth++] = m;
    x[0] = pw[0]; x[1] = pw[1]; x[2] = pw[2];
    u[0] = dw[0]; u[1] = dw[1]; u[2] = dw[2];
    for (int l = depth - 1; l >= 0; l--) {
        const int m = path[l];
        double xl[3], ul[3];
        into_child(W, W->lv[W->parent[m]], W->slot[m], x, xl, u, ul);
        for (int k = 0; k < 3; k++) { x[k] = xl[k]; u[k] = ul[k]; }
    }
}

static int world_locate_one(const orc_world *W, const double *pw) {
    for (int k = 0; k < 3; k++)
        if (!isfinite(pw[k])) return -2;
    double buf[PBUF];
    const int v = W->root;
    if (!orc_contains(W->mkind[v], shape_block(W->mkind[v], W->mparams + 5 * v, W->pdata, buf), pw)) return -1;
    return descend(W, 0, pw);
}

/* levels of placements between the root and node, and the size of the
 * coordinates they move: |world point| + the sum of their |translation| */
static int node_depth(const orc_world *W, int node, const double *pw, double *fscale) {
    int depth = 0;
    double f = sqrt(pw[0] * pw[0] + pw[1] * pw[1] + pw[2] * pw[2]);
    for (int m = node; m > 0; m = W->parent[m]) {
        const double *t = W->trans + 3 * (W->doff[W->lv[W->parent[m]]] + W->slot[m]);
        f += sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        depth++;
    }
    *fscale = f;
    return depth;
}

static int world_step_one(const orc_world *W, int node, int blocked, const double *pw, const double *dw,
                          double *step, int *blocked_out, navres *info) {
    *blocked_out = -1;
    if (info) { info->err = 0.0; info->hit = -2; info->face = F_NONE; }
    if (node < 0 || node >= W->nnodes) { *step = NAN; return -2; }
    double x[3], u[3];
    node_frame(W, node, pw, dw, x, u);
    orc_scene s = world_scene(W, W->lv[node]);
    double fscale;
    const int depth = node_depth(W, node, pw, &fscale);
    navres r = navigate_one_f(&s, x, u, blocked == -2 || (blocked >= 0 && blocked < s.nd) ? blocked : -1, depth,
                              fscale);
    if (info) *info = r;
    *step = r.step;
    if (r.hit == -2) return -2;
    const double b[3] = { x[0] + r.step * u[0], x[1] + r.step * u[1], x[2] + r.step * u[2] };
    if (r.hit >= 0) {
        double xl[3];
        into_child(W, W->lv[node], r.hit, b, xl, NULL, NULL);
        *blocked_out = -2;
        return descend(W, W->first[node] + r.hit, xl);
    }
    double xb[3] = { b[0], b[1], b[2] };
    for (int m = node; m != 0; m = W->parent[m]) {
        const int P = W->parent[m], v = W->lv[P], left = W->slot[m];
        double xp[3];
        into_parent(W, v, left, xb, xp);
        for (int j = 0; j < W->nd[v]; j++) {
            if (j == left) continue;
            double xl[3];
            into_child(W, v, j, xp, xl, NULL, NULL);
            double buf[PBUF];
            const int o = W->doff[v] + j;
            if (orc_contains(W->kinds[o], shape_block(W->kinds[o], W->params + 5 * o, W->pdata, buf), xl)) {
                *blocked_out = -2;
                return descend(W, W->first[P] + j, xl);
            }
        }
        double buf[PBUF];
        if (orc_contains(W->mkind[v], shape_block(W->mkind[v], W->mparams + 5 * v, W->pdata, buf), xp)) {
            *blocked_out = left;
            return P;
        }
        xb[0] = xp[0]; xb[1] = xp[1]; xb[2] = xp[2];
    }
    return -1;   /* left the root */
}

#define WORLD_ARGS int nlv, const int32_t *mkind, const double *mparams, const int32_t *nd, \
                   const int32_t *doff, const int32_t *kinds, const double *params, const double *rot, \
                   const double *trans, const int32_t *child, const double *pdata, int root, int max_nodes, \
                   int32_t *t_lv, int32_t *t_parent, int32_t *t_slot, int32_t *t_first
#define MAKE_WORLD orc_world W = { nlv, mkind, mparams, nd, doff, kinds, params, rot, trans, child, pdata, root, \
                                   0, t_lv, t_parent, t_slot, t_first }

/* Node table only; returns the node count (-1 past max_nodes). */
int orc_world_nodes(WORLD_ARGS) {
    MAKE_WORLD;
    return world_nodes(&W, max_nodes);
}

int orc_world_locate(WORLD_ARGS, int64_t n, const double *px, const double *py, const double *pz,
                     int32_t *node) {
    MAKE_WORLD;
    if (world_nodes(&W, max_nodes) < 0) return -1;
    for (int64_t i = 0; i < n; i++) {
        const double pw[3] = { px[i], py[i], pz[i] };
        node[i] = world_locate_one(&W, pw);
    }
    return W.nnodes;
}

/* err, hit, face (each nullable): the step's a-priori FP64 error bound (the
 * placements down to the node included), the winner in the node's volume
 * and its surface. */
int orc_world_step(WORLD_ARGS, int64_t n, const double *px, const double *py, const double *pz,
                   const double *dx, const double *dy, const double *dz, const int32_t *node_in,
                   const int32_t *blocked_in, double *step, int32_t *node_out, int32_t *blocked_out,
                   double *err, int32_t *hit, int32_t *face) {
    MAKE_WORLD;
    if (world_nodes(&W, max_nodes) < 0) return -1;
    for (int64_t i = 0; i < n; i++) {
        const double pw[3] = { px[i], py[i], pz[i] }, dw[3] = { dx[i], dy[i], dz[i] };
        int b;
        navres r;
        node_out[i] = world_step_one(&W, node_in[i], blocked_in ? blocked_in[i] : -1, pw, dw, &step[i], &b, &r);
        if (blocked_out) blocked_out[i] = b;
        if (err) err[i] = r.err;
        if (hit) hit[i] = r.hit;
        if (face) face[i] = r.face;
    }
    return W.nnodes;
}
