// Compile-time dispatch of runtime sizes: f(std::integral_constant<int, V>{}) for the value V a
// runtime size maps to (blur height, patch half-size K, register bucket of L_s).
#pragma once
#include <type_traits>

namespace fuse {

template <typename F>
void with_bh(int bh, F&& f) {
    switch (bh) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        case 5: f(std::integral_constant<int, 5>{}); break;
        case 7: f(std::integral_constant<int, 7>{}); break;
        case 9: f(std::integral_constant<int, 9>{}); break;
        case 11: f(std::integral_constant<int, 11>{}); break;
        case 13: f(std::integral_constant<int, 13>{}); break;
        default: f(std::integral_constant<int, 15>{}); break;
    }
}

template <typename F>
void with_k(int K, F&& f) {
    switch (K) {
        case 0: f(std::integral_constant<int, 0>{}); break;
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        default: f(std::integral_constant<int, 3>{}); break;
    }
}

// MAXLS bucket of the register-resident pixel kernels (0 = the wide, shared-memory kernel).
inline int pixel_bucket(int Ls) {
    return Ls <= 4 ? 4 : Ls <= 8 ? 8 : Ls <= 16 ? 16 : Ls <= 20 ? 20 : Ls <= 32 ? 32 : 0;
}

template <typename F>
void with_maxls(int Ls, F&& f) {
    switch (pixel_bucket(Ls)) {
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        case 20: f(std::integral_constant<int, 20>{}); break;
        case 32: f(std::integral_constant<int, 32>{}); break;
        default: f(std::integral_constant<int, 0>{}); break;
    }
}

}  // namespace fuse
