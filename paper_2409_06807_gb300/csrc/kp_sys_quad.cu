// kp_sys_quad.cu -- kernels and launchers of one system (see kp_launch.cuh).
#include "kp_layout.h"
#define KP_SYS kp::KP_SYS_QUAD
// resident blocks per SM the register budget is fitted to (measured best)
#define KP_MIN_BLOCKS 3
#define KP_SYS_NAME quad
#include "kp_launch.cuh"
