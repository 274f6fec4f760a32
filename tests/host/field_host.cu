// Host build of the library's host-and-device field routines, for CPU tests:
// the divstep inversion (run on the host, the same source the kernels use)
// and the compile-time Montgomery constants of both BN254 fields.
//
//   field_host consts q|r     prints p, R mod p, R^2, R^3, (p - 1) / 2, n0, -p^-1 mod R and 2^-128 mod p
//   field_host inv q|r        reads one hex value per line, prints x^-1 mod p
//
// Values are printed as 64 hex digits, most significant word first.
#include <cstdio>
#include <cstring>

#include "field.cuh"

namespace {

void put(const uint32_t *w) {
    for (int i = 7; i >= 0; i--) std::printf("%08x", w[i]);
    std::printf("\n");
}

bool get(const char *s, uint32_t *w) {
    size_t n = std::strlen(s);
    while (n && (s[n - 1] == '\n' || s[n - 1] == '\r')) n--;
    if (n != 64) return false;
    for (int i = 0; i < 8; i++) {
        uint32_t v = 0;
        for (int k = 0; k < 8; k++) {
            const char c = s[(7 - i) * 8 + k];
            const int d = c >= '0' && c <= '9' ? c - '0' : c >= 'a' && c <= 'f' ? c - 'a' + 10 : -1;
            if (d < 0) return false;
            v = (v << 4) | (uint32_t)d;
        }
        w[i] = v;
    }
    return true;
}

template <class P>
void consts() {
    uint32_t w[8];
    for (int i = 0; i < 8; i++) w[i] = P::p(i);
    put(w);
    for (int i = 0; i < 8; i++) w[i] = P::one(i);
    put(w);
    for (int i = 0; i < 8; i++) w[i] = P::r2(i);
    put(w);
    for (int i = 0; i < 8; i++) w[i] = P::r3(i);
    put(w);
    for (int i = 0; i < 8; i++) w[i] = P::half(i);
    put(w);
    std::printf("%08x\n", P::n0);
    for (int i = 0; i < 8; i++) w[i] = P::ninv(i);
    put(w);
    for (int i = 0; i < 8; i++) w[i] = P::rinvh(i);
    put(w);
}

template <class P>
int inv() {
    uint32_t pm[8];
    for (int i = 0; i < 8; i++) pm[i] = P::p(i);
    char line[256];
    while (std::fgets(line, sizeof line, stdin)) {
        uint32_t x[8], y[8];
        if (!get(line, x)) return 2;
        zk::detail::inv_divsteps(x, pm, P::n0, y);
        put(y);
    }
    return 0;
}

}  // namespace

int main(int argc, char **argv) {
    if (argc != 3 || (std::strcmp(argv[2], "q") && std::strcmp(argv[2], "r"))) return 2;
    const bool q = argv[2][0] == 'q';
    if (!std::strcmp(argv[1], "consts")) {
        if (q) consts<zk::FqP>();
        else consts<zk::FrP>();
        return 0;
    }
    if (!std::strcmp(argv[1], "inv")) return q ? inv<zk::FqP>() : inv<zk::FrP>();
    return 2;
}
