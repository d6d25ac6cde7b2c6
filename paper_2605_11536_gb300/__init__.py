"""GB300-native ToF ReSTIR: the hot path of "ToF ReSTIR: Time-of-Flight Rendering with
Spatio-temporal Reservoir Resampling" (Kim, Jarosz, Pediredla, ACM TOG 45(4), 2026) as a C-ABI
CUDA library (libtof.so, include/tof.h) with a thin Python binding (``tof``) and seeded synthetic
scene generators (``scenes``)."""
