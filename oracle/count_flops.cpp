// count_flops.cpp -- floating-point operation count of one oracle step.
//
// TEST INFRASTRUCTURE: built and run by oracle/count_flops.py (and its test),
// never by the product path.
//
// The oracle's own source (dugks_oracle.c) is compiled here as C++ with its
// scalar type `double` replaced by CountedReal, a one-double wrapper whose
// arithmetic operators and square root add to global counters.  Nothing of
// the scheme is restated: the count is of the operations the plain oracle
// performs, stage by stage in the paper's order (Eqs. 15-19, 27-33 of
// arXiv:1810.07802), for one step of a problem other than the first.
// Negation and comparisons are not counted; +, -, *, / and sqrt count one
// each (the oracle is built without contraction, so it has no fused
// multiply-adds); sin and cos (prescribed velocity fields only) are counted
// apart.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <unordered_set>

namespace flopcount {
unsigned long long add, mul, div, sqrt_, trig;
// Distinct operations: an operation applied again to operands with the same
// values (bit for bit; + and * in either order) is a common subexpression
// that any implementation computes once, e.g. a relaxation coefficient the
// oracle recomputes for each of the nine directions.  Operations that are an
// identity or a sign change (x * 0, x * 1, x * -1, x + 0, x - 0, 0 - x, x / 1:
// a lattice velocity component times a value) are not arithmetic either and
// are left out of this count.
unsigned long long distinct;
bool track;
struct Key {
    uint64_t a, b;
    int op;
    bool operator==(const Key &o) const { return a == o.a && b == o.b && op == o.op; }
};
struct KeyHash {
    size_t operator()(const Key &k) const {
        uint64_t h = k.a * 0x9E3779B97F4A7C15ull ^ (k.b + 0x632BE59BD9B4E019ull + (h_rot(k.a)));
        return (size_t)(h ^ (uint64_t)k.op * 0xC2B2AE3D27D4EB4Full);
    }
    static uint64_t h_rot(uint64_t x) { return (x << 29) | (x >> 35); }
};
std::unordered_set<Key, KeyHash> seen;
inline uint64_t bits(double x) {
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
}
inline bool trivial(int op, double a, double b) {
    auto unit = [](double x) { return x == 0.0 || x == 1.0 || x == -1.0; };
    switch (op) {
    case 0: return a == 0.0 || b == 0.0;        // x + 0
    case 1: return a == 0.0 || b == 0.0;        // x - 0, 0 - x
    case 2: return unit(a) || unit(b);          // x * 0, x * 1, x * -1
    case 3: return b == 1.0 || b == -1.0;       // x / 1, x / -1
    default: return false;
    }
}
inline void note(int op, double a, double b, bool commutes) {
    if (!track || trivial(op, a, b)) return;
    uint64_t x = bits(a), y = bits(b);
    if (commutes && x > y) std::swap(x, y);
    if (seen.insert(Key{x, y, op}).second) distinct++;
}
}  // namespace flopcount

struct CountedReal {
    double v;
    CountedReal() = default;
    constexpr CountedReal(double x) : v(x) {}
    CountedReal &operator+=(CountedReal o) { flopcount::add++; flopcount::note(0, v, o.v, true); v += o.v; return *this; }
    CountedReal &operator-=(CountedReal o) { flopcount::add++; flopcount::note(1, v, o.v, false); v -= o.v; return *this; }
    CountedReal &operator*=(CountedReal o) { flopcount::mul++; flopcount::note(2, v, o.v, true); v *= o.v; return *this; }
    CountedReal &operator/=(CountedReal o) { flopcount::div++; flopcount::note(3, v, o.v, false); v /= o.v; return *this; }
};
static inline CountedReal operator+(CountedReal a, CountedReal b) {
    flopcount::add++;
    flopcount::note(0, a.v, b.v, true);
    return a.v + b.v;
}
static inline CountedReal operator-(CountedReal a, CountedReal b) {
    flopcount::add++;
    flopcount::note(1, a.v, b.v, false);
    return a.v - b.v;
}
static inline CountedReal operator*(CountedReal a, CountedReal b) {
    flopcount::mul++;
    flopcount::note(2, a.v, b.v, true);
    return a.v * b.v;
}
static inline CountedReal operator/(CountedReal a, CountedReal b) {
    flopcount::div++;
    flopcount::note(3, a.v, b.v, false);
    return a.v / b.v;
}
static inline CountedReal operator-(CountedReal a) { return -a.v; }
static inline bool operator<(CountedReal a, CountedReal b) { return a.v < b.v; }
static inline bool operator>(CountedReal a, CountedReal b) { return a.v > b.v; }
static inline bool operator<=(CountedReal a, CountedReal b) { return a.v <= b.v; }
static inline bool operator>=(CountedReal a, CountedReal b) { return a.v >= b.v; }
static inline bool operator==(CountedReal a, CountedReal b) { return a.v == b.v; }
static inline bool operator!=(CountedReal a, CountedReal b) { return a.v != b.v; }
static inline bool operator!(CountedReal a) { return !a.v; }
static inline CountedReal sqrt(CountedReal a) {
    flopcount::sqrt_++;
    flopcount::note(4, a.v, 0.0, false);
    return std::sqrt(a.v);
}
static inline CountedReal sin(CountedReal a) { flopcount::trig++; return std::sin(a.v); }
static inline CountedReal cos(CountedReal a) { flopcount::trig++; return std::cos(a.v); }

#define double CountedReal
#include "dugks_oracle.c"
#undef double

// One counted step (the second) of an nx x ny periodic problem: the coupled
// model on a spinodal-like field (density ratio 1000, viscosity ratio 10,
// sigma 1e-3, W 4, M 0.02), or the Allen-Cahn model with a uniform velocity.
// Prints a JSON object with the counts per cell update.
int main(int argc, char **argv) {
    const int coupled = argc > 1 ? std::atoi(argv[1]) : 1;
    const int nx = 64, ny = 64;
    oracle_params P;
    std::memset(&P, 0, sizeof P);
    P.nx = nx;
    P.ny = ny;
    P.model = coupled ? 0 : 1;
    P.cfl = 0.5;
    P.mobility = 0.02;
    P.width = 4.0;
    P.rho_h = 1000.0;
    P.rho_l = 1.0;
    P.mu_h = 10.0;
    P.mu_l = 0.1;
    P.sigma = 1e-3;
    P.u0x = 0.01;
    P.u0y = 0.01;
    const long N = (long)nx * ny;
    CountedReal *phi0 = (CountedReal *)std::malloc(sizeof(CountedReal) * N);
    unsigned long long s = 20181018ull;
    for (long k = 0; k < N; k++) {   // phi = 0.5 + 0.01 (2U - 1), U from a 64-bit LCG
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        const double U = (double)(s >> 11) * (1.0 / 9007199254740992.0);
        phi0[k] = CountedReal(0.5 + 0.01 * (2.0 * U - 1.0));
    }
    oracle_ctx *c = oracle_create(&P, phi0, nullptr, nullptr, nullptr);
    if (!c) return 1;
    oracle_step(c, 1);
    flopcount::add = flopcount::mul = flopcount::div = flopcount::sqrt_ = flopcount::trig = 0;
    flopcount::distinct = 0;
    flopcount::track = true;
    oracle_step(c, 1);
    flopcount::track = false;
    const double n = (double)N;
    const unsigned long long total = flopcount::add + flopcount::mul + flopcount::div + flopcount::sqrt_;
    std::printf("{\"model\": \"%s\", \"cells\": %ld, \"flops_per_cell\": %.3f, \"distinct_flops_per_cell\": %.3f, "
                "\"add_sub\": %.3f, \"mul\": %.3f, \"div\": %.3f, \"sqrt\": %.3f, \"sin_cos\": %.3f}\n",
                coupled ? "coupled" : "allen-cahn", N, total / n, flopcount::distinct / n, flopcount::add / n,
                flopcount::mul / n, flopcount::div / n, flopcount::sqrt_ / n, flopcount::trig / n);
    oracle_destroy(c);
    std::free(phi0);
    return 0;
}
