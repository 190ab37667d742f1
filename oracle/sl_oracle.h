/*
 * sl_oracle.h -- interface of the CPU oracle (test infrastructure only; the
 * product library never includes this header).
 */
#ifndef SL_ORACLE_H
#define SL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* field kinds and their parameter layouts: see orc_field() */
enum {
    ORC_FIELD_ZERO = 0,
    ORC_FIELD_AFFINE = 1,
    ORC_FIELD_ROTATION = 2,
    ORC_FIELD_SWIRL = 3,
    ORC_FIELD_FOURIER8 = 4,
    ORC_FIELD_PAPER = 5
};

/* per-node flags */
enum {
    ORC_FLAG_CLIPPED = 1,     /* the Euler foot left the square and was clipped */
    ORC_FLAG_DEGENERATE = 2,  /* the foot lies on an edge line of its triangle */
    ORC_FLAG_MULTI = 4,       /* more than one triangle contains the foot */
    ORC_FLAG_EXCLUDED = 8     /* exclusion mode: the Euler foot left the square (Sec. 4) */
};

typedef struct orc_mesh orc_mesh;

void orc_field(int kind, const double *p, double x, double y, double t, double *fx, double *fy);
int orc_foot(int kind, const double *p, double dt, double t, double x, double y, double *X, double *Y);
int orc_orient_sign(double ax, double ay, double bx, double by, double cx, double cy);
/* orient(a, b, q) for q = (qxh + qxl, qyh + qyl), the sum taken exactly */
int orc_orient_sign2(double ax, double ay, double bx, double by, double qxh, double qyh, double qxl, double qyl);
void orc_set_force_exact(int on);
long orc_exact_calls(void);

orc_mesh *orc_mesh_create(int64_t n, int64_t nt, const double *xy, const int32_t *tri);
void orc_mesh_destroy(orc_mesh *m);
int orc_mesh_bins(const orc_mesh *m);
int orc_locate(const orc_mesh *m, double X, double Y, int32_t *tri, int *flags);
double orc_interp(const orc_mesh *m, int32_t j, double X, double Y, const double *V);
/* orc_locate for the point (X + Xl, Y + Yl), taken exactly */
int orc_locate2(const orc_mesh *m, double X, double Y, double Xl, double Yl, int32_t *tri, int *flags);

int orc_step_range(const orc_mesh *m, int kind, const double *p, double dt, int64_t n,
                   const double *vin, double *vout, double *feet, int32_t *tri, uint8_t *flags,
                   int64_t lo, int64_t hi, int nthreads);
/* The same with exclusion (exclude != 0): a node whose Euler foot leaves the
 * square keeps V^n (vout[i] = vin[i]), tri -1, flag ORC_FLAG_EXCLUDED, feet =
 * the unclipped foot (the paper's experiments, Sec. 4). */
int orc_step_range_x(const orc_mesh *m, int kind, const double *p, double dt, int64_t n,
                     const double *vin, double *vout, double *feet, int32_t *tri, uint8_t *flags,
                     int64_t lo, int64_t hi, int nthreads, int exclude);
int orc_step(const orc_mesh *m, int kind, const double *p, double dt, int64_t n,
             const double *vin, double *vout, double *feet, int32_t *tri, uint8_t *flags,
             int nthreads);
int orc_run(const orc_mesh *m, int kind, const double *p, double dt, int64_t n0, int nsteps,
            double *v, double *scratch, int nthreads);
int orc_locate_points(const orc_mesh *m, int64_t npts, const double *q, int32_t *tri, uint8_t *flags);
/* threaded; ql (the low parts of the points) may be NULL */
int orc_locate_points2(const orc_mesh *m, int64_t npts, const double *q, const double *ql, int32_t *tri,
                       uint8_t *flags, int nthreads);
void orc_tri_signs2(const orc_mesh *m, int64_t npts, const int32_t *tri, const double *q, const double *ql,
                    int8_t *signs, int nthreads);
void orc_feet(int kind, const double *p, double dt, int64_t n, int64_t npts, const double *xy,
              double *feet, uint8_t *clipped);

#ifdef __cplusplus
}
#endif
#endif
