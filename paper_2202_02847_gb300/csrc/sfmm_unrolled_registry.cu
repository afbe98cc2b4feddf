// Registry of the compiled unrolled orders (see sfmm_unrolled_dispatch.h).
#include "sfmm_unrolled.cuh"
#include "sfmm_unrolled_dispatch.h"

// The orders with a unit per real type (sfmm_unrolled_p<P>_{f64,f32}.cu; the
// units of orders 11 and 12 are split in a batch module and a lists module,
// see sfmm_unrolled_inst.cuh).
#define SFMM_UNROLLED_ORDERS(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

namespace sfmm {
namespace unrolled {

#define SFMM_DECLARE(NS)                                                                        \
    namespace NS {                                                                              \
    bool fill(const double *, const float *);                                                   \
    bool fill_lists(const double *, const float *);                                             \
    void set_attrs(size_t);                                                                     \
    void set_attrs_lists(size_t);                                                               \
    bool batch(int, const void *const *, void *const *, const void *, long long, int,           \
               const Launch &);                                                                 \
    bool lists(int, const void *const *, const void *, const long long *, void *const *,        \
               long long, int, const Launch &);                                                 \
    }
#define SFMM_DECLARE_BOTH(P) SFMM_DECLARE(p##P##_f64) SFMM_DECLARE(p##P##_f32)
SFMM_UNROLLED_ORDERS(SFMM_DECLARE_BOTH)
#undef SFMM_DECLARE_BOTH
#undef SFMM_DECLARE

bool compiled(int P) {
    switch (P) {
#define SFMM_CASE(Q) case Q: return true;
        SFMM_UNROLLED_ORDERS(SFMM_CASE)
#undef SFMM_CASE
        default: return false;
    }
}

int table_size() { return NTAB; }

// every module's copy of the constant tables
bool fill_constants(const double *t64, const float *t32) {
    bool ok = true;
#define SFMM_FILL(P)                                                                   \
    ok = ok && p##P##_f64::fill(t64, t32) && p##P##_f64::fill_lists(t64, t32) &&      \
         p##P##_f32::fill(t64, t32) && p##P##_f32::fill_lists(t64, t32);
    SFMM_UNROLLED_ORDERS(SFMM_FILL)
#undef SFMM_FILL
    return ok;
}

void set_attributes(size_t smem) {
#define SFMM_ATTRS(P)                                                                  \
    p##P##_f64::set_attrs(smem); p##P##_f64::set_attrs_lists(smem);                    \
    p##P##_f32::set_attrs(smem); p##P##_f32::set_attrs_lists(smem);
    SFMM_UNROLLED_ORDERS(SFMM_ATTRS)
#undef SFMM_ATTRS
}

#define SFMM_CASE64(Q, CALL) case Q: return p##Q##_f64::CALL;
#define SFMM_CASE32(Q, CALL) case Q: return p##Q##_f32::CALL;

bool launch_batch(bool f64, int P, int op, const void *const *in, void *const *out,
                  const void *shift, long long count, int accumulate, const Launch &L) {
#define SFMM_B64(Q) SFMM_CASE64(Q, batch(op, in, out, shift, count, accumulate, L))
#define SFMM_B32(Q) SFMM_CASE32(Q, batch(op, in, out, shift, count, accumulate, L))
    if (f64) {
        switch (P) { SFMM_UNROLLED_ORDERS(SFMM_B64) default: break; }
    } else {
        switch (P) { SFMM_UNROLLED_ORDERS(SFMM_B32) default: break; }
    }
#undef SFMM_B64
#undef SFMM_B32
    return false;
}

bool launch_lists(bool f64, int P, int op, const void *const *src, const void *shift,
                  const long long *offsets, void *const *out, long long n_targets,
                  int accumulate, const Launch &L) {
#define SFMM_L64(Q) SFMM_CASE64(Q, lists(op, src, shift, offsets, out, n_targets, accumulate, L))
#define SFMM_L32(Q) SFMM_CASE32(Q, lists(op, src, shift, offsets, out, n_targets, accumulate, L))
    if (f64) {
        switch (P) { SFMM_UNROLLED_ORDERS(SFMM_L64) default: break; }
    } else {
        switch (P) { SFMM_UNROLLED_ORDERS(SFMM_L32) default: break; }
    }
#undef SFMM_L64
#undef SFMM_L32
    return false;
}
#undef SFMM_CASE64
#undef SFMM_CASE32

}  // namespace unrolled
}  // namespace sfmm
