// rhseg_screen_tc.cuh -- spectral-step screen for half-precision operands.
#pragma once
#include "rhseg_screen_simt.cuh"

namespace rhseg {

inline bool screen_uses_tcgen05(int precision) { (void)precision; return false; }

inline void launch_screen_tc(const LevelDev &L, int precision, int n_sm, cudaStream_t s)
{
    if (precision == 1) k_screen_simt<__half, float><<<n_sm * 2, 256, 0, s>>>(L);
    else k_screen_simt<__nv_bfloat16, float><<<n_sm * 2, 256, 0, s>>>(L);
}

}  // namespace rhseg
