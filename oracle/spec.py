"""Reads the numeric choices the paper leaves open (Sec. 2.5.2 names the
Loeffler stages and the CORDIC rotation block but gives no angles, iteration
counts or word widths) from ``include/dctgb_spec.json``.

Test infrastructure only (see the package docstring).
"""
import json
import os

_SPEC_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "include", "dctgb_spec.json")

with open(_SPEC_PATH) as _f:
    SPEC = json.load(_f)

P = int(SPEC["P_level_shift_bits"])          # fraction bits of the level-shifted input
N = int(SPEC["N_cordic_iterations"])         # CORDIC micro-rotations per rotation
R = int(SPEC["R_dequant_bits"])              # fraction bits of the dequantiser weights
QSHIFT = int(SPEC["quant_shift_bits"])       # fraction bits of the quantiser multipliers
DQ_CLAMP = int(SPEC["dequant_clamp"])        # |q * Q| is clamped to this before weighting
MAX_DEFAULT = int(SPEC["psnr_max_default"])  # MAX of Eq. 23 unless the caller asks for max(O)

ANGLE_ODD_UPPER = float(SPEC["rotations"]["odd_upper"]["angle_over_pi"])
ANGLE_ODD_LOWER = float(SPEC["rotations"]["odd_lower"]["angle_over_pi"])
ANGLE_EVEN_CORDIC = float(SPEC["rotations"]["even"]["cordic_angle_over_pi"])
