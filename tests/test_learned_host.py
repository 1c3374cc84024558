"""Host side of the learned preconditioner: the package's parameter layout and
initialisation agree with the oracle network's."""
import numpy as np

from oracle import unet_oracle as U
from paper_2310_04957_gb300 import learned


def test_layer_widths_and_parameter_count():
    assert list(learned.CONV_IN) == U.CIN and list(learned.CONV_OUT) == U.COUT
    p = learned.init_params(3)
    assert p.dtype == np.float32 and p.size == U.param_count() == 1950625


def test_initialisation_is_he_normal_with_zero_biases():
    p = learned.init_params(5).astype(np.float64)
    np.testing.assert_array_equal(p, U.init_params(5).astype(np.float32).astype(np.float64))
    o = 0
    for ci, co in zip(learned.CONV_IN, learned.CONV_OUT):
        w = p[o:o + 9 * ci * co]
        fan = 9 * (3 if ci == 16 else ci)
        assert abs(w.std() / np.sqrt(2.0 / fan) - 1.0) < 0.05
        o += 9 * ci * co
        assert (p[o:o + co] == 0).all()
        o += co
