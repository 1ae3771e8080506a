"""Seeded synthetic scene generators shared by the tests, the smoke check and the benchmark."""
from .scenes import (DESC_BIN256, DESC_F32_L2, DESC_U8_L2, Scene, config1, config2, config3,
                     config4, config5, fundamental, intrinsics, make_pair, rotation, skew,
                     uniform_pair, perturb_pose, CONFIG2_POSES, mlp_init, mlp_param_count, MLP_SIZES)
