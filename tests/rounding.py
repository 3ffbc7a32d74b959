"""Operand rounding of the tensor-core forms, written out in NumPy for the
tests: BF16 round-to-nearest-even and TF32 round-to-nearest with ties away
from zero (as the conversion instructions define them)."""
import numpy as np


def round_bf16(x):
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).reshape(np.shape(x))


def round_tf32(x):
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32).reshape(np.shape(x))


ROUND = {"bf16": round_bf16, "tf32": round_tf32}
