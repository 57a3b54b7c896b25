"""Writes soft_loss_hand.json: the soft-alignment tuning loss of two tiny pairs
worked out in closed form (no DP, no autograd), to pin oracle/softgrad.py.

Derivation (smoothed Needleman-Wunsch, every max of Eq. 1 replaced by
gamma * log-sum-exp(. / gamma); borders V(i,0) = -i p, V(0,j) = -j p):

  1 x 1 pair: three monotone paths -- the match (score s), up-then-left and
  left-then-up (each -2p):
      V = gamma ln(exp(s/g) + 2 exp(-2p/g)),  E = exp(s/g) / Z.
  1 x 2 pair: five paths -- match at (1,1) then a gap (s11 - p), a gap then
  the match at (1,2) (s12 - p), three all-gap paths (-3p each):
      Z = exp((s11-p)/g) + exp((s12-p)/g) + 3 exp(-3p/g),
      V = gamma ln Z,  E11 = exp((s11-p)/g) / Z,  E12 = exp((s12-p)/g) / Z.

Similarity s = sigmoid(w . f + b), f = [ms/ls, mt/lt, |ls-lt|/max, min/max];
gate G = sigmoid((s - thr)/tau); P = clamp(E G, eps, 1 - eps);
loss = mean over the 3 cells of -(g ln P + (1-g) ln(1-P)).

The cells are chosen so that a plausible slip changes the loss: cell (1,2)
of the second pair has E G ~ 1.6e-8 < eps (the clamp acts), the gate sign
flips every G, and a mean over pairs divides by 2 instead of 3.

Only the standard library's math is used.  Run: python tests/golden/soft_loss_hand.py
"""
import json
import math
import os

THETA = [4.0, 4.0, -2.0, 1.0, -3.0, 0.3, 0.5]  # w1..w4, b, gap, thr
GAMMA, TAU, EPS = 0.1, 0.05, 1e-7
# per pair: source length, target lengths, (ms, mt) per cell, gold per cell
PAIRS = [
    {"ls": [10], "lt": [10], "ms": [[10]], "mt": [[10]], "gold": [[1]]},
    {"ls": [10], "lt": [10, 20], "ms": [[5, 0]], "mt": [[5, 0]], "gold": [[1, 0]]},
]


def sig(x):
    return 1.0 / (1.0 + math.exp(-x))


def sim(ms, mt, ls, lt):
    w, b = THETA[:4], THETA[4]
    f = [ms / ls, mt / lt, abs(ls - lt) / max(ls, lt), min(ls, lt) / max(ls, lt)]
    return sig(sum(wi * fi for wi, fi in zip(w, f)) + b)


def main():
    p, thr, g = THETA[5], THETA[6], GAMMA
    out_pairs, total, cells = [], 0.0, 0
    for pr in PAIRS:
        s = [[sim(pr["ms"][0][j], pr["mt"][0][j], pr["ls"][0], pr["lt"][j]) for j in range(len(pr["lt"]))]]
        if len(pr["lt"]) == 1:
            z = math.exp(s[0][0] / g) + 2 * math.exp(-2 * p / g)
            E = [[math.exp(s[0][0] / g) / z]]
        else:
            a, c = math.exp((s[0][0] - p) / g), math.exp((s[0][1] - p) / g)
            z = a + c + 3 * math.exp(-3 * p / g)
            E = [[a / z, c / z]]
        V = g * math.log(z)
        G = [[sig((x - thr) / TAU) for x in s[0]]]
        P = [[min(max(e * q, EPS), 1 - EPS) for e, q in zip(E[0], G[0])]]
        bce = [[-(y * math.log(x) + (1 - y) * math.log(1 - x)) for x, y in zip(P[0], pr["gold"][0])]]
        total += sum(bce[0])
        cells += len(bce[0])
        out_pairs.append({**pr, "s": s, "V": V, "E": E, "G": G, "P": P, "bce": bce})
    doc = {"about": "soft-alignment loss of a 1x1 and a 1x2 pair in closed form (path enumeration); "
                    "see soft_loss_hand.py for the derivation",
           "theta": THETA, "gamma": GAMMA, "tau": TAU, "eps": EPS, "pairs": out_pairs, "loss": total / cells}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "soft_loss_hand.json"), "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
