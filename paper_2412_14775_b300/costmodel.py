"""The paper's abstract cost of one window (Section 3, "the reward and the penalty").

C = 1 per binary32 operation, 0.6 per binary16 operation, 0.3 per conversion between
the two; operation counts are the Cost columns of Tables 1 and 2, the DS table counted
once for the real and once for the imaginary part.  For the mixed precision of Tables
3 and 4 the conversions are s2 and s12 entering group 7 of Table 3 and the 3W
normalised terms entering group 4 of Table 4.  A reporting aid, not a timing model.
"""


def window_cost(W, mixed):
    c16 = 0.6 if mixed else 1.0
    sk = 3 * W + W + W + W + c16 * 1 + 1 + c16 * (1 + 2)
    ds = 3 * W + 3 * W + 3 * W + c16 * 3 * W + c16 * 3 + c16 * 4 + c16 * 1
    conv = (2 + 2 * 3 * W) * 0.3 if mixed else 0.0
    return sk + 2 * ds + conv
