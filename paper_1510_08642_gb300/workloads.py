"""Named workloads shared by the benchmark and the full-size parity tests.

Each is a square DD or QD product of the paper's Section 3 benchmark,
scaled to GB300: operands from inputs.uniform (leading limb U[-1, 1), lower
limbs 2^-53 U[-1/2, 1/2) below the previous one), seeds fixed here.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Workload:
    name: str
    limbs: int
    n: int
    algo: str
    cutoff: int
    seed_a: int
    seed_b: int
    slices: int = 0

    @property
    def macs(self) -> int:
        return self.n ** 3


# The headline: DD Winograd at n = 4096 (Winograd is the paper's fastest
# algorithm, Table 1), cutoff chosen by the cutoff sweep (256: four levels,
# 2401 leaves of 256^3).
DD_WINOGRAD_4096 = Workload("dd_winograd_n4096", 2, 4096, "winograd", 256, 101, 102)
DD_BLOCK_4096 = Workload("dd_block_n4096", 2, 4096, "block", 512, 101, 102)
QD_WINOGRAD_4096 = Workload("qd_winograd_n4096", 4, 4096, "winograd", 256, 103, 104)
QD_BLOCK_4096 = Workload("qd_block_n4096", 4, 4096, "block", 512, 103, 104)
# The small case the oracle finishes in well under a second (Simple, n = 128).
DD_SIMPLE_128 = Workload("dd_simple_n128", 2, 128, "simple", 512, 0, 1)
# Small cases for profiler captures: operands still larger than the L2.
DD_BLOCK_2560 = Workload("dd_block_n2560", 2, 2560, "block", 512, 105, 106)
QD_BLOCK_1536 = Workload("qd_block_n1536", 4, 1536, "block", 512, 107, 108)
DD_WINOGRAD_2560 = Workload("dd_winograd_n2560", 2, 2560, "winograd", 320, 105, 106)
# The precision study: the INT8-slice DD product against the DD Winograd
# product (integer-pipe Block leaves), n = 4096 and 8192.
DD_OZAKI_4096_S16 = Workload("dd_ozaki_n4096_s16", 2, 4096, "ozaki", 512, 101, 102, 16)
DD_OZAKI_4096_S13 = Workload("dd_ozaki_n4096_s13", 2, 4096, "ozaki", 512, 101, 102, 13)
DD_WINOGRAD_8192 = Workload("dd_winograd_n8192", 2, 8192, "winograd", 256, 109, 110)
DD_OZAKI_8192_S16 = Workload("dd_ozaki_n8192_s16", 2, 8192, "ozaki", 512, 109, 110, 16)
# Section 4 LU solve (random [-1, 1] matrix), block column K, Winograd update.
DD_LU_4096 = Workload("dd_lu_n4096", 2, 4096, "winograd", 512, 111, 0)
# The same solve with the trailing updates as INT8 residue products (CRT).
DD_LU_4096_OZ2 = Workload("dd_lu_n4096_ozaki2", 2, 4096, "ozaki2", 512, 111, 0)
# Same 256^3 leaves as the headline at n = 2048 (three levels, 343 leaves):
# operands 200 MB > L2, small enough for a counter capture; likewise QD.
DD_WINOGRAD_2048 = Workload("dd_winograd_n2048", 2, 2048, "winograd", 256, 112, 113)
QD_WINOGRAD_2048 = Workload("qd_winograd_n2048", 4, 2048, "winograd", 256, 118, 119)
DD_LU_1024 = Workload("dd_lu_n1024", 2, 1024, "winograd", 512, 114, 0)
# The CRT (Ozaki scheme II) DD product with 32 moduli (P = 113 at l = 4096).
DD_OZAKI2_4096_N32 = Workload("dd_ozaki2_n4096_n32", 2, 4096, "ozaki2", 512, 101, 102, 32)
DD_OZAKI2_8192_N32 = Workload("dd_ozaki2_n8192_n32", 2, 8192, "ozaki2", 512, 109, 110, 32)
# Section 4 QD LU solve (the paper's QD Winograd LU), n = 2048.
QD_LU_2048 = Workload("qd_lu_n2048", 4, 2048, "winograd", 256, 115, 0)
QD_LU_1024 = Workload("qd_lu_n1024", 4, 1024, "winograd", 256, 117, 0)
QD_OZAKI_4096_S32 = Workload("qd_ozaki_n4096_s32", 4, 4096, "ozaki", 512, 103, 104, 32)
# Odd order of the square sweep (odd dimensions peeled at every level).
DD_WINOGRAD_3000 = Workload("dd_winograd_n3000", 2, 3000, "winograd", 256, 120, 121)
QD_WINOGRAD_3000 = Workload("qd_winograd_n3000", 4, 3000, "winograd", 256, 122, 123)
# The CRT product with its residue products on the tcgen05 tensor cores.
DD_OZAKI2TC_4096_N32 = Workload("dd_ozaki2tc_n4096_n32", 2, 4096, "ozaki2_tc", 512, 101, 102, 32)
DD_OZAKI2TC_8192_N32 = Workload("dd_ozaki2tc_n8192_n32", 2, 8192, "ozaki2_tc", 512, 109, 110, 32)
# A capture size for the tensor-core kernel (operands and residue planes
# 0.8 GB, above the L2).
DD_OZAKI2TC_2048_N32 = Workload("dd_ozaki2tc_n2048_n32", 2, 2048, "ozaki2_tc", 512, 112, 113, 32)
DD_LU_4096_OZ2TC = Workload("dd_lu_n4096_ozaki2tc", 2, 4096, "ozaki2_tc", 512, 111, 0)
