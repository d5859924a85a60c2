/*
 * opcount.cpp -- operation count of the oracle's arithmetic.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE, like the oracle it counts: oracle.c is
 * compiled here as C++ with every double replaced by a type that counts the
 * floating-point operations performed on it, so that the algorithmic work of
 * one aircraft-step-sample (one aircraft advanced one step under one wind
 * sample in one particle, Sec. 3.3-3.6 and Sec. 7.1) is read off the oracle's
 * own loops instead of being tallied by hand.  The CUDA path never links it.
 *
 * Counting rule: every +, -, *, / and comparison of two values, every
 * minimum, maximum and absolute value, and every elementary function (sqrt,
 * exp, log, log1p, pow, sin, cos, tan, atan2, floor, fmod) counts 1; a negation and
 * a conversion count 0.  (A fused multiply-add of the CUDA path therefore
 * corresponds to 2.)  The decision-margin bookkeeping of the parity protocol
 * (orc_margin_t, ORC_MARGIN) is not part of the method and is not counted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

namespace opcount {
// one count for the library: it is built without OpenMP, so the rollout runs
// on the calling thread, and its callers count from one thread at a time
// (plain globals, no thread-local storage in a library loaded at run time)
uint64_t t_ops = 0;
int t_paused = 0;
inline void tick(uint64_t n = 1)
{
    if (!t_paused) t_ops += n;
}
}  // namespace opcount

struct cdouble {
    double v;
    cdouble() = default;
    cdouble(double x) : v(x) {}
    template <class T>
    explicit operator T() const { return (T)v; }
    cdouble &operator+=(cdouble o) { opcount::tick(); v += o.v; return *this; }
    cdouble &operator-=(cdouble o) { opcount::tick(); v -= o.v; return *this; }
    cdouble &operator*=(cdouble o) { opcount::tick(); v *= o.v; return *this; }
    cdouble &operator/=(cdouble o) { opcount::tick(); v /= o.v; return *this; }
};

inline cdouble operator+(cdouble a, cdouble b) { opcount::tick(); return cdouble(a.v + b.v); }
inline cdouble operator-(cdouble a, cdouble b) { opcount::tick(); return cdouble(a.v - b.v); }
inline cdouble operator*(cdouble a, cdouble b) { opcount::tick(); return cdouble(a.v * b.v); }
inline cdouble operator/(cdouble a, cdouble b) { opcount::tick(); return cdouble(a.v / b.v); }
inline cdouble operator-(cdouble a) { return cdouble(-a.v); }
inline bool operator<(cdouble a, cdouble b) { opcount::tick(); return a.v < b.v; }
inline bool operator<=(cdouble a, cdouble b) { opcount::tick(); return a.v <= b.v; }
inline bool operator>(cdouble a, cdouble b) { opcount::tick(); return a.v > b.v; }
inline bool operator>=(cdouble a, cdouble b) { opcount::tick(); return a.v >= b.v; }
inline bool operator==(cdouble a, cdouble b) { opcount::tick(); return a.v == b.v; }
inline bool operator!=(cdouble a, cdouble b) { opcount::tick(); return a.v != b.v; }

#define OPCOUNT_FN1(name)                                                                            \
    inline cdouble name(cdouble a) { opcount::tick(); return cdouble(::name(a.v)); }
#define OPCOUNT_FN2(name)                                                                            \
    inline cdouble name(cdouble a, cdouble b) { opcount::tick(); return cdouble(::name(a.v, b.v)); }
OPCOUNT_FN1(sqrt)
OPCOUNT_FN1(exp)
OPCOUNT_FN1(log)
OPCOUNT_FN1(log1p)
OPCOUNT_FN1(sin)
OPCOUNT_FN1(cos)
OPCOUNT_FN1(tan)
OPCOUNT_FN1(floor)
OPCOUNT_FN1(fabs)
OPCOUNT_FN2(pow)
OPCOUNT_FN2(atan2)
OPCOUNT_FN2(fmin)
OPCOUNT_FN2(fmax)
OPCOUNT_FN2(fmod)
#undef OPCOUNT_FN1
#undef OPCOUNT_FN2
inline bool isinf(cdouble a) { return ::isinf(a.v); }
inline bool isfinite(cdouble a) { return ::isfinite(a.v); }
inline bool isnan(cdouble a) { return ::isnan(a.v); }

// The margin bookkeeping: plain doubles, evaluated with the count paused.
typedef double orc_plain_double;
static inline int opcount_pause() { ++opcount::t_paused; return 0; }
static inline orc_plain_double opcount_resume(orc_plain_double v) { --opcount::t_paused; return v; }
#define ORC_MARGIN_T orc_plain_double
#define ORC_MARGIN(expr) (opcount_pause(), opcount_resume(static_cast<orc_plain_double>(expr)))

#define double cdouble
#include "oracle.c"
#undef double

extern "C" {

/* Operations counted since the last reset; reset != 0 zeroes the count. */
uint64_t orc_opcount_read(int reset)
{
    const uint64_t n = opcount::t_ops;
    if (reset) opcount::t_ops = 0;
    return n;
}

}  // extern "C"
