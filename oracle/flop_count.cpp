// FLOP-counting build of the FP64 oracle (test and measurement infrastructure
// only, like the oracle itself).
//
// sbs_oracle.c is compiled a second time as C++ with its `double` replaced by
// `counted`, a double that increments a counter for every floating-point
// operation it takes part in.  Nothing of the oracle's source changes: this
// build counts the operations of the plain statement of the method, which is
// what the roofline calls algorithmic work.  Categories:
//   add  - addition and subtraction          (1 FLOP each)
//   mul  - multiplication                    (1 FLOP each)
//   div  - division                          (1 FLOP each)
//   sqrt - square root                       (1 FLOP each)
//   fn   - exp, log, sin, cos, tan           (counted apart, not as FLOP)
// Negation, comparisons, fabs, floor, fmax and conversions are not counted.
// Operations whose operands are all literals or integers (folded constants,
// index arithmetic) are not floating-point work of the method and are not seen.
// The build is single-threaded (no OpenMP), so the counters are plain globals.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <type_traits>

namespace orc_flops {
uint64_t n_add, n_mul, n_div, n_sqrt, n_fn;
}

struct counted {
    double v;
    counted() = default;
    counted(double x) : v(x) {}
    explicit operator double() const { return v; }
    template <class T, class = typename std::enable_if<std::is_integral<T>::value>::type>
    explicit operator T() const { return (T)v; }
    counted& operator+=(counted o) { ++orc_flops::n_add; v += o.v; return *this; }
    counted& operator-=(counted o) { ++orc_flops::n_add; v -= o.v; return *this; }
    counted& operator*=(counted o) { ++orc_flops::n_mul; v *= o.v; return *this; }
    counted& operator/=(counted o) { ++orc_flops::n_div; v /= o.v; return *this; }
    friend counted operator+(counted a, counted b) { ++orc_flops::n_add; return counted(a.v + b.v); }
    friend counted operator-(counted a, counted b) { ++orc_flops::n_add; return counted(a.v - b.v); }
    friend counted operator*(counted a, counted b) { ++orc_flops::n_mul; return counted(a.v * b.v); }
    friend counted operator/(counted a, counted b) { ++orc_flops::n_div; return counted(a.v / b.v); }
    friend counted operator-(counted a) { return counted(-a.v); }
    friend counted operator+(counted a) { return a; }
    friend bool operator<(counted a, counted b) { return a.v < b.v; }
    friend bool operator>(counted a, counted b) { return a.v > b.v; }
    friend bool operator<=(counted a, counted b) { return a.v <= b.v; }
    friend bool operator>=(counted a, counted b) { return a.v >= b.v; }
    friend bool operator==(counted a, counted b) { return a.v == b.v; }
    friend bool operator!=(counted a, counted b) { return a.v != b.v; }
};

inline counted sqrt(counted a) { ++orc_flops::n_sqrt; return counted(std::sqrt(a.v)); }
inline counted exp(counted a) { ++orc_flops::n_fn; return counted(std::exp(a.v)); }
inline counted log(counted a) { ++orc_flops::n_fn; return counted(std::log(a.v)); }
inline counted sin(counted a) { ++orc_flops::n_fn; return counted(std::sin(a.v)); }
inline counted cos(counted a) { ++orc_flops::n_fn; return counted(std::cos(a.v)); }
inline counted tan(counted a) { ++orc_flops::n_fn; return counted(std::tan(a.v)); }
inline counted fabs(counted a) { return counted(std::fabs(a.v)); }
inline counted floor(counted a) { return counted(std::floor(a.v)); }
inline counted fmax(counted a, counted b) { return counted(std::fmax(a.v, b.v)); }
inline counted fmin(counted a, counted b) { return counted(std::fmin(a.v, b.v)); }
inline bool isfinite(counted a) { return std::isfinite(a.v); }
inline bool isnan(counted a) { return std::isnan(a.v); }
inline bool isinf(counted a) { return std::isinf(a.v); }

static_assert(sizeof(counted) == sizeof(double), "same layout as double");

#define double counted
extern "C" {
#include "sbs_oracle.c"
}
#undef double

extern "C" void orc_flops_reset(void)
{
    orc_flops::n_add = orc_flops::n_mul = orc_flops::n_div = orc_flops::n_sqrt = orc_flops::n_fn = 0;
}

// out = {add, mul, div, sqrt, transcendental calls}
extern "C" void orc_flops_read(uint64_t out[5])
{
    out[0] = orc_flops::n_add;
    out[1] = orc_flops::n_mul;
    out[2] = orc_flops::n_div;
    out[3] = orc_flops::n_sqrt;
    out[4] = orc_flops::n_fn;
}
