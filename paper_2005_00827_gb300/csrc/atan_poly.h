// Generated by atan_fit.py (Remez minimax fit, do not edit): atan(t) ~ t P(t^2)
// on t in [0, 1], P of degree 5, coefficients of s^0 .. s^5 rounded to FP32.
// Maximum absolute error of the FP32 evaluation over [0, 1]: 1.750e-06 rad.
#pragma once
namespace qpfrg {
constexpr float kAtanC0 = 9.999772310e-01f;
constexpr float kAtanC1 = -3.326228261e-01f;
constexpr float kAtanC2 = 1.935403794e-01f;
constexpr float kAtanC3 = -1.164264828e-01f;
constexpr float kAtanC4 = 5.264735222e-02f;
constexpr float kAtanC5 = -1.171913557e-02f;
constexpr float kAtanErr = 1.750e-06f;
}  // namespace qpfrg
