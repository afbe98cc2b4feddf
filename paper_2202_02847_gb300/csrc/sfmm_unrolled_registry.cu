// Registry of the compiled unrolled orders (see sfmm_unrolled_dispatch.h).
#include "sfmm_unrolled.cuh"
#include "sfmm_unrolled_dispatch.h"

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
SFMM_DECLARE(p6_f64)
SFMM_DECLARE(p8_f64)
SFMM_DECLARE(p10_f64)
SFMM_DECLARE(p12_f64)
SFMM_DECLARE(p6_f32)
SFMM_DECLARE(p8_f32)
SFMM_DECLARE(p10_f32)
SFMM_DECLARE(p12_f32)
#undef SFMM_DECLARE

bool compiled(int P) { return P == 6 || P == 8 || P == 10 || P == 12; }

int table_size() { return NTAB; }

// every module's copy of the constant tables (the order-12 units are split in a
// batch module and a lists module, see sfmm_unrolled_inst.cuh)
#define SFMM_FILL(NS) (NS::fill(t64, t32) && NS::fill_lists(t64, t32))
bool fill_constants(const double *t64, const float *t32) {
    return SFMM_FILL(p6_f64) && SFMM_FILL(p8_f64) && SFMM_FILL(p10_f64) && SFMM_FILL(p12_f64) &&
           SFMM_FILL(p6_f32) && SFMM_FILL(p8_f32) && SFMM_FILL(p10_f32) && SFMM_FILL(p12_f32);
}
#undef SFMM_FILL

void set_attributes(size_t smem) {
#define SFMM_ATTRS(NS) NS::set_attrs(smem); NS::set_attrs_lists(smem);
    SFMM_ATTRS(p6_f64)
    SFMM_ATTRS(p8_f64)
    SFMM_ATTRS(p10_f64)
    SFMM_ATTRS(p12_f64)
    SFMM_ATTRS(p6_f32)
    SFMM_ATTRS(p8_f32)
    SFMM_ATTRS(p10_f32)
    SFMM_ATTRS(p12_f32)
#undef SFMM_ATTRS
}

#define SFMM_PICK(P, F64, CALL)                                 \
    if (F64) {                                                  \
        switch (P) {                                            \
            case 6: return p6_f64::CALL;                        \
            case 8: return p8_f64::CALL;                        \
            case 10: return p10_f64::CALL;                      \
            case 12: return p12_f64::CALL;                      \
        }                                                       \
    } else {                                                    \
        switch (P) {                                            \
            case 6: return p6_f32::CALL;                        \
            case 8: return p8_f32::CALL;                        \
            case 10: return p10_f32::CALL;                      \
            case 12: return p12_f32::CALL;                      \
        }                                                       \
    }                                                           \
    return false;

bool launch_batch(bool f64, int P, int op, const void *const *in, void *const *out,
                  const void *shift, long long count, int accumulate, const Launch &L) {
    SFMM_PICK(P, f64, batch(op, in, out, shift, count, accumulate, L))
}

bool launch_lists(bool f64, int P, int op, const void *const *src, const void *shift,
                  const long long *offsets, void *const *out, long long n_targets,
                  int accumulate, const Launch &L) {
    SFMM_PICK(P, f64, lists(op, src, shift, offsets, out, n_targets, accumulate, L))
}
#undef SFMM_PICK

}  // namespace unrolled
}  // namespace sfmm
