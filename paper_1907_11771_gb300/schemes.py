"""Extrapolation schemes printed in the paper, as data for gbs_set_weights.

A scheme is fully specified by its dependent step counts {n_dep}, its free
step counts {n_free} and the free weights c_free (Sec. 3.7); the library
solves the dependent weights from the order constraints.  Square schemes have
no free part (Sec. 3.2).

* GBS_8_6   -- Sec. 3.8.1 (order 8, six cores, ISB_n 0.7675)
* GBS_8_8   -- Sec. 3.8.2 (order 8, eight cores, ISB_n 0.8176); the printed
               list of free step counts is one short of its 11 weights, and all
               even counts up to N_max = 30 are used (Sec. 3.6), so 24 is added.
* GBS_12_8  -- Sec. 3.8.3 (order 12, eight cores, ISB_n 0.7116)
* SQ8_TABLE1, SQ12_TABLE1, SQ16_TABLE1 -- Table 1 (fully determined)
* SQ8_2468  -- classical Richardson extrapolation with N = 2, 4, 6, 8 (order 8)
* GBS_6_6   -- order 6 on six cores (all even counts up to N_max = 22): the App. B optimum at
               order 6 kept 1e-4 inside the unit circle, rounded to rationals with denominators
               below 2^16 (as Sec. 3.8 does for its schemes; optimize.gbs_6_6_free_weights
               regenerates them); exact ISB 17.65602 (ISB_n 0.76765), order-7 error term
               nonzero.  Without the margin the order-6 optimum coincides with the order-8 one
               (ISB_n 0.7695), whose order-7 term vanishes.  The paper prints no order-6 scheme:
               square order-6 schemes have ISB 0 (Sec. 2.2).
"""
from dataclasses import dataclass
from fractions import Fraction


@dataclass(frozen=True)
class Scheme:
    name: str
    order: int
    steps_dep: tuple
    steps_free: tuple = ()
    c_free_text: tuple = ()

    @property
    def c_free(self):
        """Free weights rounded to nearest FP64."""
        return tuple(float(Fraction(t)) for t in self.c_free_text)

    @property
    def steps(self):
        return tuple(self.steps_dep) + tuple(self.steps_free)

    @property
    def m(self):
        return len(self.steps)

    @property
    def evals_per_core(self):
        """N_max + 1: function evaluations per core with pair folding (Sec. 3.6)."""
        return max(self.steps) + 1

    @property
    def updates_per_point(self):
        """Grid-point updates per macro-step: sum_k (N_k + 1) (FE plus N_k leap-frog steps)."""
        return sum(n + 1 for n in self.steps)


GBS_8_6 = Scheme("GBS_8,6", 8, (2, 4, 6, 10), (8, 12, 14, 16, 18, 20, 22),
                 ("2165/767488", "13805/611712", "4553/72080", "14503/66520", "27058/7627",
                  "-86504/5761", "40916/3367"))

GBS_8_8 = Scheme("GBS_8,8", 8, (2, 26, 28, 30), (4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 24),
                 ("6833/476577792", "10847/91078656", "15235/34643968", "383/321152", "543/198784",
                  "9947/1741056", "6243/543104", "6875/296192", "1401/28496", "17713/152688",
                  "6375/19264"))

GBS_12_8 = Scheme("GBS_12,8", 12, (2, 8, 10, 16, 24, 26), (4, 6, 12, 14, 18, 20, 22, 28, 30),
                  ("235/21030240256", "4147/1612709888", "11521/39731200", "2375/3528704",
                   "6435/708736", "1291/15780", "11311/4672", "-180864/751", "222080/2079"))

SQ8_TABLE1 = Scheme("SQ8{2,16,18,20}", 8, (2, 16, 18, 20))
SQ12_TABLE1 = Scheme("SQ12{2,8,12,14,16,20}", 12, (2, 8, 12, 14, 16, 20))
SQ16_TABLE1 = Scheme("SQ16{2,8,...,22}", 16, (2, 8, 10, 12, 14, 16, 18, 22))
SQ8_2468 = Scheme("SQ8{2,4,6,8}", 8, (2, 4, 6, 8))

GBS_6_6 = Scheme("GBS_6,6", 6, (2, 4, 6), (8, 10, 12, 14, 16, 18, 20, 22),
                 ("188/59023", "124/13615", "1361/56815", "4025/60943", "6469/28645", "90535/24952",
                  "-1002769/65522", "508409/41177"))

ALL = {s.name: s for s in (GBS_8_6, GBS_8_8, GBS_12_8, SQ8_TABLE1, SQ12_TABLE1, SQ16_TABLE1, SQ8_2468, GBS_6_6)}
