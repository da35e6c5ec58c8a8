/* FP64 oracle of the learned warm-start network (test infrastructure only).
 *
 * The network is the one the learned warm start uses: a 3-layer perceptron
 * 10 -> 128 -> 128 -> 6 with ReLU after the two hidden layers.  Inputs are the
 * per-contact features, outputs the initial multipliers and the first global
 * iterate's offset at the contact vertex.  The paper has no learned part; this
 * is the plain definition written out: dense layers, ReLU, mean-squared loss
 * L = (1/B) sum_b 0.5 |y_b - t_b|^2 and its gradient by the chain rule.
 *
 * Flat parameter layout: W1[128][10] b1[128] W2[128][128] b2[128] W3[6][128] b3[6].
 * Parity: pinned against central finite differences of the loss.
 */
#include <stdlib.h>
#include <string.h>

#define NI 10
#define NH 128
#define NO 6

static void layout(const double *p, const double **W1, const double **b1, const double **W2,
                   const double **b2, const double **W3, const double **b3) {
  *W1 = p; *b1 = *W1 + NH * NI; *W2 = *b1 + NH; *b2 = *W2 + NH * NH; *W3 = *b2 + NH; *b3 = *W3 + NO * NH;
}

static void forward_one(const double *p, const double *x, double *h1, double *h2, double *y) {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
  layout(p, &W1, &b1, &W2, &b2, &W3, &b3);
  for (int i = 0; i < NH; i++) {
    double s = b1[i];
    for (int j = 0; j < NI; j++) s += W1[i * NI + j] * x[j];
    h1[i] = s > 0 ? s : 0;
  }
  for (int i = 0; i < NH; i++) {
    double s = b2[i];
    for (int j = 0; j < NH; j++) s += W2[i * NH + j] * h1[j];
    h2[i] = s > 0 ? s : 0;
  }
  for (int i = 0; i < NO; i++) {
    double s = b3[i];
    for (int j = 0; j < NH; j++) s += W3[i * NH + j] * h2[j];
    y[i] = s;
  }
}

void or_mlp_forward(int B, const double *p, const double *x, double *y) {
  double h1[NH], h2[NH];
  for (int b = 0; b < B; b++) forward_one(p, x + NI * b, h1, h2, y + NO * b);
}

double or_mlp_loss_grad(int B, const double *p, const double *x, const double *t, double *grad) {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
  layout(p, &W1, &b1, &W2, &b2, &W3, &b3);
  int np = NH * NI + NH + NH * NH + NH + NO * NH + NO;
  memset(grad, 0, sizeof(double) * np);
  double *gW1 = grad, *gb1 = gW1 + NH * NI, *gW2 = gb1 + NH, *gb2 = gW2 + NH * NH, *gW3 = gb2 + NH,
         *gb3 = gW3 + NO * NH;
  double h1[NH], h2[NH], y[NO], dy[NO], d2[NH], d1[NH], loss = 0;
  for (int b = 0; b < B; b++) {
    const double *xb = x + NI * b, *tb = t + NO * b;
    forward_one(p, xb, h1, h2, y);
    for (int i = 0; i < NO; i++) {
      double e = y[i] - tb[i];
      loss += 0.5 * e * e / B;
      dy[i] = e / B;
    }
    for (int i = 0; i < NO; i++) {
      gb3[i] += dy[i];
      for (int j = 0; j < NH; j++) gW3[i * NH + j] += dy[i] * h2[j];
    }
    for (int j = 0; j < NH; j++) {
      double s = 0;
      for (int i = 0; i < NO; i++) s += W3[i * NH + j] * dy[i];
      d2[j] = h2[j] > 0 ? s : 0;
    }
    for (int i = 0; i < NH; i++) {
      gb2[i] += d2[i];
      for (int j = 0; j < NH; j++) gW2[i * NH + j] += d2[i] * h1[j];
    }
    for (int j = 0; j < NH; j++) {
      double s = 0;
      for (int i = 0; i < NH; i++) s += W2[i * NH + j] * d2[i];
      d1[j] = h1[j] > 0 ? s : 0;
    }
    for (int i = 0; i < NH; i++) {
      gb1[i] += d1[i];
      for (int j = 0; j < NI; j++) gW1[i * NI + j] += d1[i] * xb[j];
    }
  }
  return loss;
}
